"""Checks of the shared synthetic-input generator (not the method)."""
import numpy as np

from synthetic.phantom import (WORKLOADS, make_workload, pals_dmu, pals_mu,
                               smooth_heaviside, smooth_heaviside_deriv)


def test_smooth_heaviside_is_compact_and_c1():
    s = np.linspace(-0.5, 0.5, 2001)
    H = smooth_heaviside(s)
    assert np.all(H[s <= -0.15] == 0) and np.all(H[s >= 0.15] == 1)
    fd = np.gradient(H, s)
    assert np.max(np.abs(fd - smooth_heaviside_deriv(s))) < 1e-3


def test_dmu_matches_finite_differences():
    inp = make_workload("t3d_12")
    p = inp["params"][1]
    X = inp["X"]
    dmu = pals_dmu(p, X, 0.01)
    for k in range(p.size):
        d = 1e-7 * max(1, abs(p[k]))
        e = np.zeros_like(p); e[k] = d
        fd = (pals_mu(p + e, X, 0.01) - pals_mu(p - e, X, 0.01)) / (2 * d)
        assert np.max(np.abs(fd - dmu[k])) <= 1e-5 * max(1.0, np.abs(dmu[k]).max())


def test_workload_shapes_and_seeding():
    a = make_workload("t2d_37")
    b = make_workload("t2d_37")
    assert np.array_equal(a["mu"], b["mu"])
    wl = a["wl"]
    assert a["mu"].shape == (wl.K + 1, wl.n) and a["D"].shape == (wl.n,)
    assert len(a["src_nodes"]) == wl.nsrc and len(a["det_nodes"]) == wl.ndet
    assert np.all(a["D"] > 0) and np.all(a["mu"] >= 0.01 - 1e-15)
    assert WORKLOADS["c2_3d64"].n == 64 ** 3 and WORKLOADS["c3_3d128"].n == 2097152
    assert WORKLOADS["c5_3d192"].n == 7077888


def test_grid_support_route_gives_the_same_fields():
    """pals_mu / pals_dmu on the node grid: the index-box route (grid=...)
    and the plain per-point route give identical arrays, also for anomalies
    that touch the domain boundary."""
    from synthetic.phantom import node_coords, node_grid
    for name in ("t3d_21", "t2d_37"):
        wl = WORKLOADS[name]
        X = node_coords(wl)
        rng = np.random.default_rng(12)
        d = wl.dim
        p = np.zeros((3, d + 2))
        p[:, :d] = rng.uniform(0.0, 1.0, size=(3, d))
        p[0, :d] = 0.02                                   # centre outside the node range
        p[:, d] = rng.uniform(0.05, 0.2, size=3)
        p[:, d + 1] = 0.03
        p = p.ravel()
        assert np.array_equal(pals_mu(p, X, 0.01), pals_mu(p, X, 0.01, node_grid(wl)))
        assert np.array_equal(pals_dmu(p, X, 0.01), pals_dmu(p, X, 0.01, node_grid(wl)))


def test_training_phantoms_draw_two_to_six_anomalies_from_the_seed_law():
    """The learned network's training phantoms (C4: random 2-6-anomaly
    phantoms): each vector holds n_a (d + 2) parameters with n_a in 2..6,
    centres in [0.15, 0.85], widths in [0.05, 0.15], absorptions in
    [0.02, 0.05]; seeded (the same call gives the same phantoms) and not
    jitters of the workload's phantom."""
    import numpy as np
    from synthetic.phantom import WORKLOADS, training_params, seed_params
    wl = WORKLOADS["c4_3d128"]
    ps = training_params(wl, 40)
    d = wl.dim
    counts = set()
    for p in ps:
        q = np.asarray(p).reshape(-1, d + 2)
        counts.add(q.shape[0])
        assert 2 <= q.shape[0] <= 6
        assert np.all((q[:, :d] >= 0.15) & (q[:, :d] <= 0.85))
        assert np.all((q[:, d] >= 0.05) & (q[:, d] <= 0.15))
        assert np.all((q[:, d + 1] >= 0.02) & (q[:, d + 1] <= 0.05))
    assert counts == {2, 3, 4, 5, 6}
    again = training_params(wl, 40)
    assert all(np.array_equal(a, b) for a, b in zip(ps, again))
    p0 = seed_params(wl, np.random.default_rng(wl.seed)).reshape(-1, d + 2)
    assert not any(np.asarray(p).size == p0.size and np.allclose(np.asarray(p).reshape(-1, d + 2)[:, :d], p0[:, :d],
                                                                 atol=0.1) for p in ps)
