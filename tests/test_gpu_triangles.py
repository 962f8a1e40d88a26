"""Triangle-union quadrature (Sec. 4.3, the Koch snowflake) on the GPU: the
TRIANGLES family's nodes and fields against the oracle's own triangle rule
and direct sum."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_05978_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def plan(*a, **k):
    from paper_2010_05978_gb300 import Plan
    return Plan(*a, **k)


BARS = {"fp64": (1e-12, 1e-10), "fp32": (1e-6, 1e-6)}


def test_triangle_nodes_match_oracle():
    fams = W.koch_families(2, 0.05)
    fams[1] = dict(fams[1], cx=0.2, cy=-0.1)
    p = plan(fams, 0.05, 1.0, 1e-6, grid=W.grid_spec(64, 64, 0.05))
    x, y, w = (t.cpu().numpy() for t in p.nodes())
    ox, oy, ow = (np.concatenate(v) for v in zip(*[Q.family_nodes(f) for f in fams]))
    assert len(x) == len(ox) == sum(len(f["tri"]) * f["p"] ** 2 for f in fams)
    assert np.max(np.abs(x - ox)) < 5e-15 and np.max(np.abs(y - oy)) < 5e-15
    assert np.max(np.abs(w - ow)) < 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_koch_t1_grid(prec):
    """Level-3 snowflake at lz = 0.02 (p = 109, 37, 13, 5 by level) on a 128^2
    grid over [-1.5, 1.5)^2."""
    fams = W.koch_families(3, 0.02)
    g = W.grid_spec(128, 128, 3.0 / 128)
    xi, eta = oracle.grid_targets(128, 128, 3.0 / 128)
    ref = oracle.field(fams, 0.02, 1.0, xi, eta, output="occulter").reshape(128, 128)
    tol, bar = BARS[prec]
    u = plan(fams, 0.02, 1.0, tol, precision=prec, grid=g, output="occulter").eval()
    assert rel_l2(u.cpu().numpy(), ref) <= bar


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_triangles_t3_scattered(prec):
    """Random, translated triangles of either orientation (negative areas
    subtract) at scattered targets."""
    g = W.rng(46, 0)
    tri = g.uniform(-0.8, 0.8, (40, 6))
    fam = [{"kind": "triangles", "tri": tri, "p": 12, "cx": 0.1, "cy": -0.05},
           dict(W.koch_families(1, 0.05)[1], cx=-0.2)]
    xi, eta = W.disc_targets(3000, 1.3, 47)
    ref = oracle.field(fam, 0.05, 1.0, xi, eta)
    tol, bar = BARS[prec]
    p = plan(fam, 0.05, 1.0, tol, precision=prec, box=(-1.3, 1.3, -1.3, 1.3))
    u = p.eval(torch.tensor(np.stack([xi, eta], 1), device="cuda")).cpu().numpy()
    assert rel_l2(u, ref) <= bar


def test_koch_L13_full_size_sampled():
    """The bench's workload at full size (level 13: 67.1M triangles, 67.2M
    nodes, FP32 fast mode, 1000^2 grid at lz = 0.01): sampled grid targets
    against the oracle's direct sum over its own snowflake rule."""
    fams = W.koch_families(13, 0.01)
    g = W.grid_spec(1000, 1000, 0.003)
    u = plan(fams, 0.01, 1.0, 1e-6, precision="fp32", grid=g, output="occulter",
             recompute_nodes=True).eval().cpu().numpy().ravel()
    xi, eta = oracle.grid_targets(1000, 1000, 0.003)
    sel = W.rng(48, 0).choice(1_000_000, 12, replace=False)
    ref = oracle.field(fams, 0.01, 1.0, xi[sel], eta[sel], output="occulter")
    assert rel_l2(u[sel], ref) <= 1e-6
