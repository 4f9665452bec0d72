"""Given their workspaces, ot_spread (sorted), ot_interpolate (trilinear, whose cell means need
scratch) and ot_field_subtract_mean allocate nothing: after ten calls of each, the default
stream-ordered memory pool has seen no allocation (its used-memory high-water mark stays at
zero) and the device's free memory is unchanged.  Results stay bitwise identical call to
call."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POOL_RESERVED_HIGH, POOL_USED_HIGH = 6, 8  # cudaMemPoolAttr values (driver_types.h)


def _cudart():
    """The CUDA runtime the library is linked against (already loaded in this process)."""
    for line in open("/proc/self/maps"):
        path = line.split()[-1]
        if "libcudart.so" in path:
            return C.CDLL(path)
    pytest.skip("libcudart not mapped")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import synth
    ot._L()
    rt = _cudart()
    w = synth.tiny()
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    return torch, ot, rt, w, tree


def _pool(rt, torch):
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), torch.cuda.current_device()) == 0
    return pool


def _pool_attr(rt, pool, attr):
    v = C.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, attr, C.byref(v)) == 0
    return v.value


def _free_bytes(rt):
    free, total = C.c_size_t(), C.c_size_t()
    assert rt.cudaMemGetInfo(C.byref(free), C.byref(total)) == 0
    return free.value


@pytest.mark.parametrize("mates", [False, True])
def test_calls_allocate_nothing_given_workspace(env, mates):
    torch, ot, rt, w, tree = env
    ot.ot_octree_build_mates(tree, mates)
    n_leaves = ot.ot_octree_info(tree)[0]
    dev = "cuda"
    X = [torch.as_tensor(np.ascontiguousarray(w.markers[d]), device=dev) for d in range(3)]
    P = [torch.as_tensor(np.ascontiguousarray(w.particles[d]), device=dev) for d in range(3)]
    F = torch.as_tensor(np.ascontiguousarray(w.forces, dtype=np.float32), device=dev)
    rng = np.random.default_rng(3)
    field = torch.as_tensor(rng.normal(size=(n_leaves, 4)).astype(np.float32), device=dev)
    fld = field.clone()
    # every output and workspace exists before the counted calls
    ws_s = torch.empty(ot.ot_spread_workspace_size(tree, ot.OT_PESKIN4, X[0].numel()), dtype=torch.uint8, device=dev)
    ws_i = torch.empty(ot.ot_interpolate_workspace_size(tree, ot.OT_TRILINEAR), dtype=torch.uint8, device=dev)
    ws_m = torch.empty(ot.ot_field_mean_workspace_size(tree), dtype=torch.uint8, device=dev)
    f = torch.zeros((n_leaves, 4), dtype=torch.float32, device=dev)
    u = torch.empty((3, P[0].numel()), dtype=torch.float32, device=dev)
    um = torch.empty((3, X[0].numel()), dtype=torch.float32, device=dev)
    mean = torch.empty(3, dtype=torch.float64, device=dev)
    refs = None

    def calls():
        f.zero_()
        ot.ot_spread(tree, ot.OT_PESKIN4, ot.OT_SORTED, X[0], X[1], X[2], F, f, workspace=ws_s)
        ot.ot_interpolate(tree, ot.OT_TRILINEAR, P[0], P[1], P[2], field, u=u, workspace=ws_i)
        ot.ot_interpolate(tree, ot.OT_PESKIN4, X[0], X[1], X[2], field, u=um)
        fld.copy_(field)
        ot.ot_field_subtract_mean(tree, fld, mean=mean, workspace=ws_m)

    calls()  # first use: lazy module loading and kernel attribute queries happen here
    torch.cuda.synchronize()
    refs = [t.clone() for t in (f, u, um, fld, mean)]
    pool = _pool(rt, torch)
    zero = C.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, POOL_USED_HIGH, C.byref(zero)) == 0
    assert rt.cudaMemPoolSetAttribute(pool, POOL_RESERVED_HIGH, C.byref(zero)) == 0
    used0 = _pool_attr(rt, pool, POOL_USED_HIGH)
    free0 = _free_bytes(rt)
    for _ in range(10):
        calls()
    torch.cuda.synchronize()
    assert _pool_attr(rt, pool, POOL_USED_HIGH) == used0 == 0
    assert _free_bytes(rt) == free0
    for a, b in zip((f, u, um, fld, mean), refs):
        assert torch.equal(a, b)


def test_short_workspace_is_refused(env):
    torch, ot, rt, w, tree = env
    P = [torch.as_tensor(np.ascontiguousarray(w.particles[d][:64]), device="cuda") for d in range(3)]
    n_leaves = ot.ot_octree_info(tree)[0]
    field = torch.zeros((n_leaves, 4), dtype=torch.float32, device="cuda")
    need = ot.ot_interpolate_workspace_size(tree, ot.OT_TRILINEAR)
    assert need > 0 and ot.ot_interpolate_workspace_size(tree, ot.OT_PESKIN4) == 0
    assert ot.ot_interpolate_workspace_size(tree, ot.OT_TRILINEAR, fp64=True) > need
    short = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ot.OtError):
        ot.ot_interpolate(tree, ot.OT_TRILINEAR, *P, field, workspace=short)
    with pytest.raises(ot.OtError):
        ot.ot_field_subtract_mean(tree, field, workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
