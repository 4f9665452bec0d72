"""ot_spread_noalloc through the C ABI: the sorted spreading variant for callers that cannot
allocate device memory (its scratch is the library's fixed device array).  Its output must equal
the allocating ot_spread(OT_SORTED) bit for bit on two calls in a row (the same per-leaf sums in
the same marker order), match the FP64 oracle within the FP32 tolerance, accept exactly the
documented maximum marker counts and refuse one more before anything is launched.  This file
is collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
MAX_MARKERS = {2: 150_635, 3: 508_394}  # the limits stated in include/octtrack.h


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import synth
    lib = C.CDLL(ot.library_path())
    fn = lib.ot_spread_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                   C.c_void_p, C.c_void_p]
    w = synth.tiny()
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    return torch, ot, fn, w, tree


def _call(torch, fn, tree, kernel, X, F, dV, f):
    p = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(tree.handle, kernel, p(X[0]), p(X[1]), p(X[2]), p(F), p(dV), X[0].numel(), p(f), s)


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("with_dv", [False, True])
def test_noalloc_matches_sorted_spread_twice(env, kernel, with_dv):
    import oracle
    torch, ot, fn, w, tree = env
    n_leaves = ot.ot_octree_info(tree)[0]
    rng = np.random.default_rng(41)
    X = [torch.as_tensor(np.ascontiguousarray(w.markers[d]), device="cuda") for d in range(3)]
    n = X[0].numel()
    F = torch.as_tensor(rng.normal(size=(3, n)).astype(np.float32), device="cuda")
    dV = None
    if with_dv:
        dV = torch.as_tensor((rng.uniform(0.5, 2.0, n) * 2.0 ** (-3 * w.lmax)).astype(np.float32), device="cuda")
    ref = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
    ot.ot_spread(tree, kernel, ot.OT_SORTED, X[0], X[1], X[2], F, ref, dV=dV)
    for _ in range(2):
        f = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
        assert _call(torch, fn, tree, kernel, X, F, dV, f) == 0
        torch.cuda.synchronize()
        assert torch.equal(f, ref)
    # and against the FP64 oracle on the same inputs
    ko, lo = oracle.octree_build(w.spheres, w.lmin, w.lmax)
    f_ref, _ = oracle.spread_delta(ko, lo, w.lmax, kernel, *w.markers, F.double().cpu().numpy(),
                                   dV=None if dV is None else dV.double().cpu().numpy())
    scale = float(np.abs(f_ref[:, :3]).max())
    assert float(np.abs(f.cpu().numpy()[:, :3] - f_ref[:, :3]).max()) <= TOL32 * scale
    assert torch.all(f[:, 3] == 0)


@pytest.mark.parametrize("kernel", [2, 3])
def test_noalloc_limit_is_exact(env, kernel):
    """The documented maximum runs (and equals the allocating spreading); one more marker is
    refused with OT_ERR_LIMIT and leaves the output untouched."""
    torch, ot, fn, w, tree = env
    n_leaves = ot.ot_octree_info(tree)[0]
    m = MAX_MARKERS[kernel]
    reps = -(-m // w.markers.shape[1])
    Xh = np.tile(w.markers, reps)[:, :m + 1]
    X = [torch.as_tensor(np.ascontiguousarray(Xh[d]), device="cuda") for d in range(3)]
    F = torch.as_tensor(np.random.default_rng(5).normal(size=(3, m + 1)).astype(np.float32), device="cuda")
    f = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
    over = _call(torch, fn, tree, kernel, X, F, None, f)
    torch.cuda.synchronize()
    assert over == -8 and torch.count_nonzero(f) == 0
    Xm = [x[:m].contiguous() for x in X]
    Fm = F[:, :m].contiguous()
    assert _call(torch, fn, tree, kernel, Xm, Fm, None, f) == 0
    ref = torch.zeros_like(f)
    ot.ot_spread(tree, kernel, ot.OT_SORTED, Xm[0], Xm[1], Xm[2], Fm, ref)
    torch.cuda.synchronize()
    assert torch.equal(f, ref)


def test_noalloc_refuses_sizes_beyond_its_scratch(env):
    torch, ot, fn, w, tree = env
    x = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")
    F = torch.zeros((3, 1), dtype=torch.float32, device="cuda")
    f = torch.zeros((4,), dtype=torch.float32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many = 10_000_000  # far beyond the fixed scratch; refused before any launch
    assert fn(tree.handle, 2, p(x), p(x), p(x), p(F), None, too_many, p(f), s) == -8
    assert fn(tree.handle, 1, p(x), p(x), p(x), p(F), None, 1, p(f), s) == -1  # trilinear has no spreading


@pytest.mark.parametrize("case", ["one_block", "small_1", "small_2", "small_33", "with_coarse"])
def test_noalloc_and_sorted_agree_on_run_edge_cases(env, case):
    """The allocating sorted spreading splits the sorted pairs into equal shares per warp and
    deals the parent-block runs that start in each share to its lanes; the allocation-free one
    reduces fixed chunks with the weights recomputed.  They must agree bit for bit where that
    split is stressed -- runs far longer than a warp's share (20,000 markers on one spot:
    every pair in the same few blocks), fewer pairs than warps (1, 2, 33 markers), and pairs
    of blocks that are not refined to the finest level (sorted last, dropped) -- and both must
    match the oracle."""
    import oracle
    torch, ot, fn, w, tree = env
    n_leaves = ot.ot_octree_info(tree)[0]
    rng = np.random.default_rng(7)
    m0 = w.markers[:, :1]
    if case == "one_block":
        Xh = m0 + rng.uniform(-1e-7, 1e-7, (3, 20000))
    elif case.startswith("small_"):
        Xh = w.markers[:, :int(case.split("_")[1])]
    else:  # a third of the markers near a corner of the cube, where the tree is coarse
        Xh = np.concatenate([w.markers[:, :600], rng.uniform(0.0, 0.05, (3, 300))], axis=1)
    Xh = np.ascontiguousarray(Xh)
    X = [torch.as_tensor(np.ascontiguousarray(Xh[d]), device="cuda") for d in range(3)]
    n = Xh.shape[1]
    F = torch.as_tensor(rng.normal(size=(3, n)).astype(np.float32), device="cuda")
    ref = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
    ot.ot_spread(tree, 2, ot.OT_SORTED, X[0], X[1], X[2], F, ref)
    f = torch.zeros_like(ref)
    assert _call(torch, fn, tree, 2, X, F, None, f) == 0
    torch.cuda.synchronize()
    assert torch.equal(f, ref)
    ot.ot_last_error(tree, clear=True)
    ko, lo = oracle.octree_build(w.spheres, w.lmin, w.lmax)
    f_ref, bad = oracle.spread_delta(ko, lo, w.lmax, 2, *Xh, F.double().cpu().numpy())
    assert (bad > 0) == (case == "with_coarse")
    scale = float(np.abs(f_ref[:, :3]).max())
    assert float(np.abs(ref.cpu().numpy()[:, :3] - f_ref[:, :3]).max()) <= TOL32 * scale


def test_noalloc_and_sorted_agree_with_many_runs_per_warp(env):
    """150,000 markers scattered through the single bubble's finest shell: about 2M pairs in
    short runs, hundreds of runs per warp share, so the allocating reduce sorts each batch of run
    heads by length before dealing it to the lanes.  Bit for bit against the allocation-free
    reduce, which splits the same pairs into fixed chunks instead."""
    torch, ot, fn, _, _ = env
    from paper_2605_20565_gb300 import synth
    wb = synth.single_bubble(n_markers=10, n_particles=10)
    tree = ot.ot_octree_build(wb.spheres, wb.lmin, wb.lmax)
    n_leaves = ot.ot_octree_info(tree)[0]
    c, r, shell = wb.spheres[0, :3], wb.spheres[0, 3], wb.spheres[0, 4]
    rng = np.random.default_rng(11)
    n = 150_000
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    Xh = np.ascontiguousarray(c[:, None] + d * (r + rng.uniform(-0.4, 0.4, n) * shell))
    assert np.all((Xh > 0) & (Xh < 1))
    X = [torch.as_tensor(np.ascontiguousarray(Xh[k]), device="cuda") for k in range(3)]
    F = torch.as_tensor(rng.normal(size=(3, n)).astype(np.float32), device="cuda")
    ref = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
    ot.ot_spread(tree, 2, ot.OT_SORTED, X[0], X[1], X[2], F, ref)
    f = torch.zeros_like(ref)
    assert _call(torch, fn, tree, 2, X, F, None, f) == 0
    torch.cuda.synchronize()
    assert torch.equal(f, ref)
    assert ot.ot_last_error(tree) & ot.OT_DEV_STENCIL == 0
    assert float(ref[:, :3].abs().sum()) > 0
