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


CHECK_STEPS = (0, 1, 9, 10, 11, 50, 99)


@pytest.mark.parametrize("search", [0, 1])
def test_tracking_per_step_parity(env, search):
    """Steps 0, 1, 9, 10, 11, 50 and 99 of a 100-step run with re-adaptation every 10 steps (map
    level 8, level-mate and parent-block tables, value records), each checked against the
    oracle on inputs the oracle side makes itself: the octree rebuilt from the moved spheres
    (bit for bit); the batch and the single-op calls at the oracle's own particle trajectory
    (FP64 AB2 driven by its own interpolation) and at the markers' rigidly moved positions, with
    the workload's field at the oracle's leaf centres in FP32 on both sides (hosts bit for bit,
    values within 1e-5); the sorted spreading; one GPU AB2 step from the oracle's state."""
    torch, ot, synth, tracking, w = env
    w = synth.tracking(seed=4, n_particles=20000, lmax=9, n_bubbles=64)
    h = 2.0 ** -w.lmax
    centres0, vel = w.extra["centres"], w.extra["velocities"]
    radii, shells = 0.5 * w.extra["diameters"], w.spheres[:, 4]

    def spheres(t):
        return np.column_stack([centres0 + vel * t, radii, shells])

    def oracle_side(t):
        ko, lo = oracle.octree_build(spheres(t), w.lmin, w.lmax)
        f32 = synth.fourier_field(w.modes, oracle.leaf_centres(ko, lo)).astype(np.float32)
        return ko, lo, f32

    ko, lo, f32 = oracle_side(0.0)
    dt = h / float(np.abs(f32[:, :3]).max())
    re_coef = 2.0
    tr = tracking.Tracker(w, search=search, rebuild_every=10, map_level=8, mates=True, dt=dt, re_coef=re_coef,
                          n_leaf_models=4096, n_mid_models=64)
    assert ot.ot_octree_get_map_level(tr.tree) == 8 and ot.ot_octree_has_mates(tr.tree)
    P = w.particles
    st = {"x": P.copy(), "v": np.zeros_like(P), "a_prev": np.zeros_like(P), "v_prev": np.zeros_like(P)}
    t = 0.0
    n_m = w.markers.shape[1]
    dev = torch.device("cuda")
    F32 = np.ascontiguousarray(w.forces, dtype=np.float32)
    checked = 0
    for step in range(100):
        if step % 10 == 0 and step > 0:
            ko, lo, f32 = oracle_side(t)
        host = oracle.locate_ub(ko, lo, *st["x"])
        u_ref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *st["x"], host)
        if step in CHECK_STEPS:
            checked += 1
            assert tr.tree_step == step - step % 10 and tr.step_no == step
            k, l = ot.ot_octree_copy_leaves(tr.tree)
            assert np.array_equal(k.cpu().numpy().view(np.uint64), ko) and np.array_equal(l.cpu().numpy(), lo)
            fld = torch.as_tensor(f32, device=dev)
            scale = float(np.abs(f32[:, :3]).max())
            M = tr.markers_at(t)
            um_ref, bad = oracle.interp_delta(ko, lo, w.lmax, 2, f32.astype(np.float64), *M)
            assert bad == 0
            f_ref, _ = oracle.spread_delta(ko, lo, w.lmax, 2, *M, F32.astype(np.float64))
            x = [torch.as_tensor(np.ascontiguousarray(st["x"][d]), device=dev) for d in range(3)]
            m = [torch.as_tensor(np.ascontiguousarray(M[d]), device=dev) for d in range(3)]
            up = torch.empty((3, P.shape[1]), dtype=torch.float32, device=dev)
            um = torch.empty((3, n_m), dtype=torch.float32, device=dev)
            hp = torch.empty(P.shape[1], dtype=torch.int32, device=dev)
            hm = torch.empty(n_m, dtype=torch.int32, device=dev)
            b = ot.ot_batch_create(tr.tree, [dict(kernel=ot.OT_PESKIN4, x=m[0], y=m[1], z=m[2], u=um, host=hm),
                                             dict(kernel=ot.OT_TRILINEAR, x=x[0], y=x[1], z=x[2], u=up, host=hp)],
                                   fld, search=search, launch=tr.launch)
            ot.ot_batch_run(b)
            u1 = ot.ot_interpolate(tr.tree, ot.OT_TRILINEAR, *x, fld, search=search)
            fs = torch.zeros_like(fld)
            ot.ot_spread(tr.tree, ot.OT_PESKIN4, ot.OT_SORTED, *m, torch.as_tensor(F32, device=dev), fs)
            torch.cuda.synchronize()
            del b
            assert np.array_equal(hp.cpu().numpy(), host)
            assert np.array_equal(hm.cpu().numpy(), oracle.locate_ub(ko, lo, *M))
            assert np.abs(up.cpu().numpy() - u_ref).max() <= 1e-5 * scale
            assert torch.equal(up, u1)
            assert np.abs(um.cpu().numpy() - um_ref).max() <= 1e-5 * scale
            assert np.abs(fs[:, :3].cpu().numpy() - f_ref[:, :3]).max() <= 1e-5 * np.abs(f_ref[:, :3]).max()
            # one AB2 step on the device from the oracle's state and velocities
            xs = torch.as_tensor(st["x"], device=dev).contiguous()
            vs, a0, v0 = [torch.as_tensor(st[key].astype(np.float32), device=dev) for key in ("v", "a_prev", "v_prev")]
            ot.ot_advect_ab2(xs, vs, a0, v0, torch.as_tensor(u_ref.astype(np.float32), device=dev), tr.tau, re_coef,
                             dt, first=step == 0, periodic=True)
        oracle.advect_ab2(st, u_ref, tr.tau, re_coef, dt, step == 0, periodic=True)
        if step in CHECK_STEPS:
            torch.cuda.synchronize()
            vscale = max(float(np.abs(st["v"]).max()), 1e-30)
            assert np.abs(vs.cpu().numpy() - st["v"]).max() <= 1e-5 * vscale
            dx = np.abs(xs.cpu().numpy() - st["x"])
            assert np.minimum(dx, 1.0 - dx).max() <= 1e-9
        tr.step()
        t += dt
        assert tr.t == t  # the same time on both sides: the spheres of each re-adaptation agree
    torch.cuda.synchronize()
    assert checked == len(CHECK_STEPS)
    # the GPU's own trajectory stays valid (FP32 and FP64 trajectories diverge: not compared)
    x = tr.x.cpu().numpy()
    assert np.all(np.isfinite(x)) and np.all((x >= 0) & (x < 1))
    assert ot.ot_last_error(tr.tree) & (ot.OT_DEV_STENCIL | ot.OT_DEV_OUTSIDE) == 0
