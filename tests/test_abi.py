"""CPU checks of the C ABI: the library loads, exports every symbol that
include/*.h declares, and validates its arguments on the host (no device work)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1603_09577_gb300 import _lib as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|const char \*|void)\s*\**\s*(lbm3?_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = C.lib()
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(C.declared_symbols()) <= set(names) | {"lbm_last_error"}


def desc(**kw):
    d = C.Desc()
    d.nx, d.ny, d.prec, d.bc_x, d.bc_y = 16, 12, C.LBM_F32, 0, 0
    d.steps_per_pass, d.per_cell_K = 1, 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def ws_size(d):
    n = ctypes.c_size_t()
    rc = C.lib().lbm_workspace_size(ctypes.byref(d), ctypes.byref(n))
    return rc, n.value


def test_workspace_size_and_layout():
    rc, n32 = ws_size(desc())
    assert rc == 0
    # two buffers of 9 planes, rows padded to 64 elements
    assert n32 >= 2 * 9 * 12 * 64 * 4
    rc, n64 = ws_size(desc(prec=C.LBM_F64))
    assert rc == 0 and n64 > n32
    rc, nb = ws_size(desc(prec=C.LBM_BF16S))
    assert rc == 0 and nb < n32
    rc, nk = ws_size(desc(per_cell_K=1))
    assert rc == 0 and nk > n32
    rc, _ = ws_size(desc(steps_per_pass=2))
    assert rc == 0
    rc, _ = ws_size(desc(steps_per_pass=2, prec=C.LBM_F64))
    assert rc == C.LBM_EUNSUPPORTED


@pytest.mark.parametrize("bad", [dict(nx=1), dict(ny=0), dict(prec=7), dict(bc_x=3), dict(steps_per_pass=3),
                                 dict(block_rows=16), dict(block_rows=3), dict(kernel_variant=5), dict(kernel_variant=6),
                                 dict(kernel_variant=3), dict(kernel_variant=4)])
def test_invalid_descriptions_rejected(bad):
    rc, _ = ws_size(desc(**bad))
    assert rc == C.LBM_EINVAL
    assert C.lib().lbm_last_error()


class FakeWorkspace:
    """A host buffer that stands in for the device workspace: lbm_create only
    records pointers, and the tests below make no device calls."""

    def __init__(self, n):
        self.buf = ctypes.create_string_buffer(n + 512)
        a = ctypes.addressof(self.buf)
        self.ptr = (a + 255) & ~255


def make(d=None):
    d = d or desc()
    rc, n = ws_size(d)
    ws = FakeWorkspace(n)
    h = ctypes.c_void_p()
    assert C.lib().lbm_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(ws.ptr), n) == 0
    return h, ws


def coeffs(**kw):
    c = C.Coeffs()
    c.conv, c.diff = 0, 0
    c.u[:] = [0.05, 0.02]
    c.K[:] = [0.01, 0.0, 0.01]
    c.s[:] = [1.0, 1.2, 1.2, 0.0, 1.0, 0.0, 1.0, 1.1, 1.1]
    for k, v in kw.items():
        if k in ("u", "K", "s", "Dm"):
            getattr(c, k)[:] = v
        else:
            setattr(c, k, v)
    return c


def test_create_rejects_bad_workspace():
    d = desc()
    rc, n = ws_size(d)
    ws = FakeWorkspace(n)
    h = ctypes.c_void_p()
    L = C.lib()
    assert L.lbm_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(ws.ptr + 8), n) == C.LBM_EINVAL
    assert L.lbm_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(ws.ptr), n - 1) == C.LBM_EINVAL
    assert L.lbm_create(ctypes.byref(h), ctypes.byref(d), None, n) == C.LBM_EINVAL


@pytest.mark.parametrize("bad", [
    dict(K=[0.01, 0.02, 0.01]),         # not positive definite
    dict(K=[-0.01, 0.0, 0.01]),
    dict(s=[1.0, 2.5, 1.2, 0, 1, 0, 1, 1.1, 1.1]),
    dict(s=[1.0, 1.2, 0.0, 0, 1, 0, 1, 1.1, 1.1]),
    dict(conv=5), dict(diff=-1), dict(r1=2.0), dict(u=[float("nan"), 0.0])])
def test_coefficient_validation(bad):
    h, ws = make()
    L = C.lib()
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(**bad))) == C.LBM_EINVAL
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs())) == 0
    L.lbm_destroy(h)


def test_calls_in_wrong_order_are_rejected_before_any_device_work():
    h, ws = make()
    L = C.lib()
    assert L.lbm_step(h, 1, None) == C.LBM_EINVAL          # no coefficients
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs())) == 0
    assert L.lbm_step(h, 1, None) == C.LBM_EINVAL          # no initial phi
    assert L.lbm_set_phi(h, None, C.LBM_F64, None) == C.LBM_EINVAL
    assert L.lbm_step(None, 1, None) == C.LBM_EINVAL
    assert b"lbm_set_phi" in L.lbm_last_error() or L.lbm_last_error()
    L.lbm_destroy(h)


def test_per_cell_field_required():
    h, ws = make(desc(per_cell_K=1))
    L = C.lib()
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(K=[0.0, 0.0, 0.0]))) == 0
    assert L.lbm_set_phi(h, ctypes.c_void_p(16), C.LBM_F64, None) == C.LBM_EINVAL
    assert b"K_field" in L.lbm_last_error()
    L.lbm_destroy(h)


@pytest.mark.parametrize("bad,code", [
    (dict(bc_x=C.LBM_NEE, bc_y=C.LBM_ABB), C.LBM_EINVAL),          # extrapolation beside an anti-bounce-back axis
    (dict(bc_x=C.LBM_NEE, nx=2), C.LBM_EINVAL),                    # no inward neighbour
    (dict(scheme=2), C.LBM_EINVAL),
    (dict(scheme=C.LBM_SCHEME_A, prec=C.LBM_BF16S), C.LBM_EUNSUPPORTED),
    (dict(bc_y=C.LBM_NEE, steps_per_pass=2, per_cell_K=1), C.LBM_EUNSUPPORTED),
    (dict(scheme=C.LBM_SCHEME_A, steps_per_pass=2, prec=C.LBM_BF16S), C.LBM_EUNSUPPORTED),
    (dict(scheme=C.LBM_SCHEME_A, kernel_variant=2), C.LBM_EUNSUPPORTED)])
def test_general_path_descriptions(bad, code):
    rc, _ = ws_size(desc(**bad))
    assert rc == code


def test_scheme_a_workspace_holds_the_phi_plane():
    _, n = ws_size(desc())
    _, na = ws_size(desc(scheme=C.LBM_SCHEME_A))
    assert na >= n + 2 * 12 * 64 * 4            # one float plane per buffer
    _, n64 = ws_size(desc(prec=C.LBM_F64))
    _, na64 = ws_size(desc(prec=C.LBM_F64, scheme=C.LBM_SCHEME_A))
    assert na64 >= n64 + 2 * 12 * 64 * 8


def test_general_path_coefficients():
    L = C.lib()
    h, ws = make(desc(scheme=C.LBM_SCHEME_A, bc_x=C.LBM_NEE))
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=2, power=2, src_family=1, b=0.1))) == 0
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=2, power=0))) == C.LBM_EINVAL
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(src_family=1, power=1, b=0.1, r1=0.2))) == C.LBM_EINVAL
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(src_family=2))) == C.LBM_EINVAL
    arr = (ctypes.c_double * 64)()
    assert L.lbm_set_dirichlet(h, ctypes.cast(arr, ctypes.c_void_p), 0) == C.LBM_EINVAL
    assert L.lbm_set_dirichlet(h, ctypes.cast(arr, ctypes.c_void_p), 1) == 0
    L.lbm_destroy(h)
    h, ws = make(desc())                               # Scheme B, periodic
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(src_family=1, power=1, b=0.1))) == C.LBM_EINVAL
    assert L.lbm_set_dirichlet(h, ctypes.cast(arr, ctypes.c_void_p), 1) == C.LBM_EINVAL
    h2, ws2 = make(desc(prec=C.LBM_BF16S))
    assert L.lbm_set_coeffs(h2, ctypes.byref(coeffs(conv=2, power=1))) == C.LBM_EUNSUPPORTED
    L.lbm_destroy(h)
    L.lbm_destroy(h2)


def test_cfree_and_buckley_leverett_coefficients():
    L = C.lib()
    h, ws = make(desc(scheme=C.LBM_SCHEME_A))
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=3, cfree=1))) == 0
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=3))) == C.LBM_EINVAL       # conv 3 needs cfree
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=1, cfree=2))) == C.LBM_EINVAL
    L.lbm_destroy(h)
    h, ws = make(desc())                                                          # Scheme B
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=0, cfree=1))) == C.LBM_EINVAL
    L.lbm_destroy(h)


def test_tensor_diffusion_coefficients():
    L = C.lib()
    h, ws = make(desc())
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(diff=3, Dm=[1.0, 1.0, 2.0]))) == 0
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(diff=4))) == C.LBM_EINVAL
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(diff=3, Dm=[float("inf"), 0.0, 1.0]))) == C.LBM_EINVAL
    L.lbm_destroy(h)
    h, ws = make(desc(steps_per_pass=2))                       # the general two-step kernel
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(diff=3, Dm=[1.0, 0.0, 1.0]))) == 0
    L.lbm_destroy(h)
    h, ws = make(desc(steps_per_pass=2, kernel_variant=3))     # the column march has no general form
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(diff=3, Dm=[1.0, 0.0, 1.0]))) == C.LBM_EUNSUPPORTED
    L.lbm_destroy(h)
    h, ws = make(desc(steps_per_pass=2, scheme=C.LBM_SCHEME_A))
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=2, power=1, src_family=1, b=0.1))) == 0
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=3, cfree=1))) == C.LBM_EUNSUPPORTED
    assert L.lbm_set_coeffs(h, ctypes.byref(coeffs(conv=1, cfree=1))) == C.LBM_EUNSUPPORTED
    L.lbm_destroy(h)


def test_d3q19_descriptions_and_coefficients():
    L = C.lib()

    def d3(**kw):
        d = C.Desc3()
        d.nx, d.ny, d.nz, d.prec = 12, 10, 8, C.LBM_F32
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    n = ctypes.c_size_t()
    assert L.lbm3_workspace_size(ctypes.byref(d3()), ctypes.byref(n)) == 0
    assert n.value >= 2 * 19 * 10 * 8 * 64 * 4
    assert L.lbm3_workspace_size(ctypes.byref(d3(prec=C.LBM_BF16S)), ctypes.byref(n)) == 0
    for bad in (dict(nz=1), dict(prec=7), dict(block_rows=3)):
        assert L.lbm3_workspace_size(ctypes.byref(d3(**bad)), ctypes.byref(n)) == C.LBM_EINVAL
    # node indices within a plane are 32-bit: rows padded to 64 elements, so
    # 2 x 1024 x 32768 nodes (2^26) make a plane of 2^31 elements, one too many
    assert L.lbm3_workspace_size(ctypes.byref(d3(nx=2, ny=1024, nz=32767)), ctypes.byref(n)) == 0
    assert L.lbm3_workspace_size(ctypes.byref(d3(nx=2, ny=1024, nz=32768)), ctypes.byref(n)) == C.LBM_EINVAL
    walled = d3()
    walled.bc[:] = [1, 0, 1]
    walled.phi_wall[:] = [0.1, 0.2, 0.0, 0.0, 0.5, 0.6]
    assert L.lbm3_workspace_size(ctypes.byref(walled), ctypes.byref(n)) == 0
    walled.bc[1] = 2                                        # extrapolation is not built in 3-D
    assert L.lbm3_workspace_size(ctypes.byref(walled), ctypes.byref(n)) == C.LBM_EINVAL
    walled.bc[1] = 0
    walled.phi_wall[3] = float("nan")
    assert L.lbm3_workspace_size(ctypes.byref(walled), ctypes.byref(n)) == C.LBM_EINVAL
    d = d3()
    L.lbm3_workspace_size(ctypes.byref(d), ctypes.byref(n))
    ws = FakeWorkspace(n.value)
    h = ctypes.c_void_p()
    assert L.lbm3_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(ws.ptr), n.value) == 0
    c = C.Coeffs3()
    c.K[:] = [0.02, 0.004, 0.002, 0.015, 0.003, 0.01]
    c.se, c.s0 = 1.1, 1.0
    assert L.lbm3_set_coeffs(h, ctypes.byref(c)) == 0
    c.K[:] = [0.02, 0.03, 0.0, 0.015, 0.0, 0.01]            # not positive definite
    assert L.lbm3_set_coeffs(h, ctypes.byref(c)) == C.LBM_EINVAL
    c.K[:] = [0.02, 0.0, 0.0, 0.02, 0.0, 0.02]
    c.se = 2.0
    assert L.lbm3_set_coeffs(h, ctypes.byref(c)) == C.LBM_EINVAL
    assert L.lbm3_step(h, 1, None) == C.LBM_EINVAL           # no initial phi
    assert L.lbm3_save(h, ctypes.c_void_p(16), None) == C.LBM_EINVAL   # nothing to save yet
    assert L.lbm3_load(h, None, None) == C.LBM_EINVAL
    sb = ctypes.c_size_t()
    assert L.lbm3_state_bytes(h, ctypes.byref(sb)) == 0
    assert sb.value == (19 * 10 * 8 * 64 * 4 + 255) // 256 * 256       # 19 planes, x pitch 64
    L.lbm3_destroy(h)
    db = d3(prec=C.LBM_BF16S)
    L.lbm3_workspace_size(ctypes.byref(db), ctypes.byref(n))
    wb = FakeWorkspace(n.value)
    assert L.lbm3_create(ctypes.byref(h), ctypes.byref(db), ctypes.c_void_p(wb.ptr), n.value) == 0
    assert L.lbm3_state_bytes(h, ctypes.byref(sb)) == 0
    plane = 10 * 8 * 64
    assert sb.value == (19 * plane * 2 + 255) // 256 * 256 + (plane * 4 + 255) // 256 * 256   # + the shift plane
    L.lbm3_destroy(h)


def test_grids_beyond_the_index_range_are_rejected():
    """Node offsets are 32-bit in places: grids above 2^31 nodes are refused on the host."""
    assert ws_size(desc(nx=65536, ny=32769))[0] == C.LBM_EINVAL
    assert ws_size(desc(nx=46340, ny=46340))[0] == 0            # 2.147e9 nodes: the largest square that fits
    d = C.Desc3()
    d.nx, d.ny, d.nz, d.prec = 2048, 1024, 1025, C.LBM_F32
    n = ctypes.c_size_t()
    assert C.lib().lbm3_workspace_size(ctypes.byref(d), ctypes.byref(n)) == C.LBM_EINVAL


def ens_sizes(pairs):
    n = len(pairs)
    return n, (ctypes.c_int * n)(*[a for a, _ in pairs]), (ctypes.c_int * n)(*[b for _, b in pairs])


def test_ensemble_host_validation():
    """The ensemble's workspace size (tables, tile partials of the per-instance
    reductions, populations) and every argument check of lbm_ensemble_create
    that runs before device work; calls on a null ensemble are rejected."""
    L = C.lib()
    n = ctypes.c_size_t()
    cnt, nx, ny = ens_sizes([(64, 40), (33, 70)])
    assert L.lbm_ensemble_workspace_size(cnt, nx, ny, ctypes.byref(n)) == C.LBM_OK
    pops = sum(2 * (((9 * ((a + 31) // 32 * 32) * b * 4) + 255) // 256 * 256) for a, b in [(64, 40), (33, 70)])
    tiles = 2 * 5 + 2 * 9                           # 32 x 8 tiles of the two instances
    assert n.value >= pops + 64 * tiles
    for bad in ([(1, 40)], [(64, 1)]):
        c, x, y = ens_sizes(bad)
        assert L.lbm_ensemble_workspace_size(c, x, y, ctypes.byref(n)) == C.LBM_EINVAL
    assert L.lbm_ensemble_workspace_size(0, nx, ny, ctypes.byref(n)) == C.LBM_EINVAL
    assert L.lbm_ensemble_workspace_size(cnt, None, ny, ctypes.byref(n)) == C.LBM_EINVAL
    assert L.lbm_ensemble_workspace_size(cnt, nx, ny, ctypes.byref(n)) == C.LBM_OK
    ws = FakeWorkspace(n.value)
    e = ctypes.c_void_p()

    def create(cs, ptr=ws.ptr, size=n.value):
        arr = (C.Coeffs * len(cs))(*cs)
        return L.lbm_ensemble_create(ctypes.byref(e), cnt, nx, ny, arr, ctypes.c_void_p(ptr), size, None)

    good = coeffs(diff=1)
    assert create([good, good], ptr=ws.ptr + 8) == C.LBM_EINVAL               # misaligned workspace
    assert create([good, good], size=n.value - 1) == C.LBM_EINVAL             # too small
    assert create([good, coeffs(diff=2)]) == C.LBM_EINVAL                      # mixed families
    assert create([good, coeffs(diff=1, s=[1.0, 2.0, 1.2, 0.0, 1.0, 0.0, 1.0, 1.1, 1.1])]) == C.LBM_EINVAL
    assert create([good, coeffs(diff=1, K=[0.01, 0.02, 0.01])]) == C.LBM_EINVAL
    assert create([good, coeffs(diff=1, r1=0.1)]) == C.LBM_EUNSUPPORTED       # no source terms
    assert create([good, coeffs(diff=1, cfree=1)]) == C.LBM_EUNSUPPORTED
    assert create([coeffs(conv=2), coeffs(conv=2)]) == C.LBM_EINVAL           # families 0-1 only
    out = ctypes.c_void_p(16)
    assert L.lbm_ensemble_step(None, 1, 0, None) == C.LBM_EINVAL
    assert L.lbm_ensemble_reduce(None, None, out, None) == C.LBM_EINVAL
    assert L.lbm_ensemble_get_phi(None, out, C.LBM_F64, None) == C.LBM_EINVAL
    assert L.lbm_ensemble_set_phi(None, out, C.LBM_F64, None) == C.LBM_EINVAL
    assert L.lbm_ensemble_replay(None, None) == C.LBM_EINVAL
    assert L.lbm_ensemble_configure(None, 2) == C.LBM_EINVAL


def test_error_messages_are_per_thread():
    """Two host threads calling failing entry points at the same time each read
    back their own message (lbm_last_error is thread-local), with no GPU work."""
    import threading
    L = C.lib()
    results = {}
    barrier = threading.Barrier(2)

    def worker(tag, bad):
        barrier.wait()
        seen = []
        for _ in range(200):
            n = ctypes.c_size_t()
            rc = L.lbm_workspace_size(ctypes.byref(bad), ctypes.byref(n))
            seen.append((rc, L.lbm_last_error()))
        results[tag] = seen

    a = desc(nx=1)                        # nx < 2
    b = desc(steps_per_pass=3)            # invalid steps per pass
    t1 = threading.Thread(target=worker, args=("a", a))
    t2 = threading.Thread(target=worker, args=("b", b))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert all(rc == C.LBM_EINVAL and b"nx and ny" in m for rc, m in results["a"])
    assert all(rc == C.LBM_EINVAL and b"steps_per_pass" in m for rc, m in results["b"])


def test_probe_and_ensemble_tile_arguments_checked_on_the_host():
    """Argument checks of lbm_probe_fp64 and lbm_ensemble_set_tiles /
    lbm_ensemble_set_persistent run before any device work."""
    L = C.lib()
    n = ctypes.c_longlong(-1)
    sink = ctypes.c_void_p(16)
    for bad in ((0, 256, 10, sink), (8, 100, 10, sink), (8, 2048, 10, sink), (8, 256, 0, sink), (8, 256, 10, None)):
        assert L.lbm_probe_fp64(*bad, ctypes.byref(n), None) == C.LBM_EINVAL, bad
    assert n.value == -1
    assert L.lbm_ensemble_set_tiles(None, 1) == C.LBM_EINVAL
    assert L.lbm_ensemble_set_persistent(None, 2) == C.LBM_EINVAL
