"""CPU checks of the seeded input recipes (workloads.py): the sizes and
structure the benches and the full-size tests rely on."""
import numpy as np

import workloads as W


def test_koch_snowflake_levels_and_node_count():
    """Sec. 4.3: level k adds 3 * 4^(k-1) triangles of side sqrt(3)/3^k; with
    p_k = max(1, ceil(s_k / (0.8 lz))) at lz = 0.01 the largest triangle gets
    p = 217 and level 13 has 67.2M nodes (the paper: about 69 million)."""
    fams = W.koch_families(8, 0.01)           # levels 9..13 only add p = 1 triangles
    assert [len(f["tri"]) for f in fams] == [1] + [3 * 4 ** (k - 1) for k in range(1, 9)]
    assert fams[0]["p"] == 217 and all(f["p"] == 1 for f in fams[5:])
    n = sum(len(f["tri"]) * f["p"] ** 2 for f in fams) + sum(3 * 4 ** (k - 1) for k in range(9, 14))
    assert n == 67_184_800
    # each level's triangles have the level's side length
    for k, f in enumerate(fams[:6]):
        t = np.asarray(f["tri"]).reshape(-1, 3, 2)
        side = np.hypot(*(t[:, 1] - t[:, 0]).T)
        assert np.allclose(side, np.sqrt(3.0) / 3.0 ** k, rtol=1e-12)


def test_random_star_batch_sizes():
    """32 instances, 1e5..2e6 nodes and 1e5..1e7 targets each, 5.5e7 targets
    in all, F_i = 1000 sqrt(N_i / 1e7)."""
    probs, counts = W.random_star_batch()
    assert len(probs) == 32 and len(counts) == 32
    assert sum(counts) == 54_885_723
    assert min(counts) >= 100_000 and max(counts) <= 10_000_000


def test_starshade_sweep_sizes():
    """64 wavelengths in [400, 1000] nm; per-wavelength node counts 14,040 to
    24,960 (uneven); the 512 x 512 pupil grid with h = 2.4 / 512."""
    cfg = W.starshade_sweep()
    lams = [q["lam"] for q in cfg["problems"]]
    assert len(lams) == 64 and np.isclose(lams[0], 400e-9) and np.isclose(lams[-1], 1000e-9)
    ns = []
    for q in cfg["problems"]:
        f = q["families"][0]
        ns.append(f["n_petals"] * f["n_p"] * f["m"] + f["n_d"] * f["m_d"])
    assert min(ns) == 14_040 and max(ns) == 24_960
    g = cfg["grid"]
    assert (g["n1"], g["n2"]) == (512, 512) and np.isclose(g["h"], 2.4 / 512)


def test_seeded_inputs_repeat():
    a = W.disc_targets(1000, 1.5, 2)
    b = W.disc_targets(1000, 1.5, 2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert np.max(np.hypot(*a)) <= 1.5
