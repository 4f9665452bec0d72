"""ot_spread_noalloc through the C ABI: the sorted spreading variant for callers that cannot
allocate device memory (its scratch is the library's fixed device array).  Its output must
match the allocating ot_spread(OT_SORTED) on two calls in a row, and sizes beyond the fixed
scratch must be refused before anything is launched.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


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
    scale = float(ref[:, :3].abs().max())
    for _ in range(2):
        f = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
        assert _call(torch, fn, tree, kernel, X, F, dV, f) == 0
        torch.cuda.synchronize()
        assert float((f - ref).abs().max()) <= TOL32 * scale
        assert torch.all(f[:, 3] == 0)


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
