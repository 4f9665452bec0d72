"""Time-stepped tracking (moving bubbles, AB2 particles, periodic re-adaptation) on the GPU.

Parity is taken on inputs that do not come from the CUDA path: the octree rebuilt at each
re-adaptation is compared bit for bit with the oracle's octree of the same moved spheres,
the re-sampled field with the field evaluated at the oracle's leaf centres, and the first
step (from the synthetic initial state) with the oracle's interpolation and AB2 update.
Later states are checked by invariants only (trajectories of FP32 and FP64 diverge)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _morton(P):
    """Morton keys of the finest (level 21) cells of points (3, n) in [0, 1)."""
    q = np.floor(np.asarray(P) * 2.0 ** 21).astype(np.uint64)
    key = np.zeros(q.shape[1], np.uint64)
    for b in range(21):
        for d in range(3):
            key |= ((q[d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return key


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import synth, tracking
    w = synth.tracking(seed=4, n_particles=20000, lmax=7, n_bubbles=16)
    return torch, ot, synth, tracking, w


def test_tracking_rebuilds_match_oracle_and_state_stays_valid(env):
    torch, ot, synth, tracking, w = env
    tr = tracking.Tracker(w, search=ot.OT_LEARNED, rebuild_every=4, n_leaf_models=2048, n_mid_models=64)
    for step in range(12):
        if step % 4 == 0:
            sph = tr.spheres_now()
            ko, lo = oracle.octree_build(sph, w.lmin, w.lmax)
            k, l = ot.ot_octree_copy_leaves(tr.tree)
            assert np.array_equal(k.cpu().numpy().view(np.uint64), ko)
            assert np.array_equal(l.cpu().numpy(), lo)
            ref = synth.fourier_field(w.modes, oracle.leaf_centres(ko, lo))
            assert np.abs(tr.field.double().cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
        tr.step()
        torch.cuda.synchronize()
        x = tr.x.cpu().numpy()
        assert np.all(np.isfinite(x)) and np.all((x >= 0) & (x < 1))
        assert torch.isfinite(tr.u).all() and torch.isfinite(tr.um).all()
        assert ot.ot_last_error(tr.tree) & (ot.OT_DEV_STENCIL | ot.OT_DEV_OUTSIDE | ot.OT_DEV_REFINED_CAP) == 0
    assert tr.timings["rebuilds"] == 4


def test_tracking_first_step_matches_oracle(env):
    torch, ot, synth, tracking, w = env
    tr = tracking.Tracker(w, search=ot.OT_BINARY, rebuild_every=100, n_leaf_models=2048, n_mid_models=64,
                          re_coef=2.0)
    ko, lo = oracle.octree_build(tr.spheres_now(), w.lmin, w.lmax)
    f32 = synth.fourier_field(w.modes, oracle.leaf_centres(ko, lo)).astype(np.float32).astype(np.float64)
    P = w.particles
    host = oracle.locate_ub(ko, lo, *P)
    u_ref = oracle.interp_trilinear(ko, lo, f32, *P, host)
    um_ref, bad = oracle.interp_delta(ko, lo, w.lmax, 2, f32, *w.markers)
    assert bad == 0
    st = {"x": P.copy(), "v": np.zeros((3, P.shape[1])), "a_prev": np.zeros((3, P.shape[1])),
          "v_prev": np.zeros((3, P.shape[1]))}
    oracle.advect_ab2(st, u_ref, tr.tau, 2.0, tr.dt, True, periodic=True)
    tr.step()
    torch.cuda.synchronize()
    # the tracker stores its particles in Morton order; ids maps them to the input order
    ids = tr.ids.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(P.shape[1]))
    assert np.all(np.diff(_morton(P[:, ids]) >> np.uint64(3 * (21 - 8))) >= 0)  # level-8 cells in order
    scale = np.abs(f32[:, :3]).max()
    assert np.abs(tr.u.cpu().numpy() - u_ref[:, ids]).max() <= 1e-5 * scale
    mids = tr.m_ids.cpu().numpy()
    assert np.array_equal(np.sort(mids), np.arange(w.markers.shape[1]))
    assert np.abs(tr.um.cpu().numpy() - um_ref[:, mids]).max() <= 1e-5 * scale
    assert np.abs(tr.v.cpu().numpy() - st["v"][:, ids]).max() <= 1e-5 * max(np.abs(st["v"]).max(), 1e-30)
    dx = np.abs(tr.x.cpu().numpy() - st["x"][:, ids])
    dx = np.minimum(dx, 1.0 - dx)  # periodic distance
    assert dx.max() <= 1e-9
    # markers moved rigidly with their bubbles
    moved = w.markers + (w.extra["velocities"][w.marker_group] * tr.dt).T
    assert np.abs(tr.mx.cpu().numpy() - moved[:, mids]).max() <= 1e-12
