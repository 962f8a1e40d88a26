"""The spreading stage's one device-side wait is bounded.

A tile holding more records than one work item takes is split into chunks
that run on several SMs: the tile's first chunk clears it and raises a ready
flag, the others wait for that flag before adding into the tile.  The wait
polls at most fresnel_opts.max_spin times; with no polls allowed every such
wait gives up at once, the evaluation reports FRESNEL_ERR_TIMEOUT and the
plan (and the device) stay usable.  With the default bound the field is the
oracle's within tol."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_05978_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _star():
    # 128 x 16 x 64 = 131,072 nodes: the spokes meet in the centre tiles,
    # which hold far more records than one chunk
    return W.star(n_panels=128, p=16, m=64, n=200)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_split_tile_wait_gives_up_with_no_polls(prec):
    from paper_2010_05978_gb300 import FresnelError, Plan
    cfg = _star()
    fam, g = cfg["families"], cfg["grid"]
    tol = 1e-6 if prec == "fp32" else 1e-12
    bad = Plan(fam, cfg["lam"], cfg["z"], tol, precision=prec, grid=g, recompute_nodes=True,
               max_spin=-1)
    for _ in range(2):   # the flags are reset by every launch: it gives up again
        with pytest.raises(FresnelError) as e:
            bad.eval()
        assert e.value.status == -4, e.value
        assert "max_spin" in str(e.value)
    bad.close()
    import oracle
    good = Plan(fam, cfg["lam"], cfg["z"], tol, precision=prec, grid=g, recompute_nodes=True)
    u = good.eval().cpu().numpy().ravel()
    xi, eta = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    idx = W.rng(2, 17).choice(len(xi), 300, replace=False)
    ref = oracle.field(fam, cfg["lam"], cfg["z"], xi[idx], eta[idx])
    bar = 1e-6 if prec == "fp32" else 1e-10
    assert np.linalg.norm(u[idx] - ref) / np.linalg.norm(ref) <= bar
