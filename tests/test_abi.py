"""The C ABI library loads and exports every function include/sfft.h declares.

No GPU: only host-side entry points are called (status strings, unknown counts).
"""
import ctypes

import pytest

import oracle
from paper_2109_09334_gb300 import binding
from paper_2109_09334_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return binding.library()


def test_exports_every_declared_symbol(lib):
    names = binding.declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/sfft.h but not exported"


def test_status_strings(lib):
    for code in range(-8, 1):
        s = binding.status_string(code)
        assert isinstance(s, str) and s
    assert binding.status_string(-4).startswith("normal matrix")


@pytest.mark.parametrize("w0,w1,dk,db,cpr", [(4, 4, 0, 0, 1), (6, 6, 1, 1, 0), (8, 8, 2, 2, 1),
                                             (8, 8, 2, 2, 0), (0, 0, 3, 3, 1), (1, 3, 2, 1, 1)])
def test_num_unknowns_matches_oracle(lib, w0, w1, dk, db, cpr):
    cfg = binding.make_config(64, 64, w0, w1, dk, db, cpr)
    assert binding.sfft_num_unknowns(cfg) == oracle.num_unknowns(oracle.OracleConfig(64, 64, w0, w1, dk, db, cpr))


def test_num_unknowns_rejects_negative(lib):
    cfg = binding.make_config(64, 64, -1, 2, 0, 0, 1)
    with pytest.raises(binding.SfftError) as e:
        binding.sfft_num_unknowns(cfg)
    assert e.value.status == binding.SFFT_ERR_INVALID


def test_struct_layouts(lib):
    assert ctypes.sizeof(binding.sfft_config) == 14 * 4
    assert ctypes.sizeof(binding.sfft_solve_info) == 24


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The product path has no fallback: without the CUDA library it raises."""
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        binding.library()


def test_unknown_counts_match_the_oracle(lib):
    """sfft_num_unknowns (no GPU use) for polynomial and B-spline bases equals
    the oracle's count of the same configuration."""
    import oracle
    cases = [((16, 16, 2, 2, 2, 2, 1), None), ((16, 16, 3, 1, 1, 0, 0), None),
             ((16, 16, 2, 2, 0, 0, 1), (2, 1, 1, 0)), ((16, 16, 1, 3, 0, 0, 0), (3, 2, 2, 3)),
             ((16, 16, 0, 0, 0, 0, 1), (0, 0, 0, 0))]
    for (n0, n1, w0, w1, dk, db, cpr), spline in cases:
        cfg = binding.make_config(n0, n1, w0, w1, dk, db, cpr, spline=spline)
        oc = oracle.OracleConfig(n0, n1, w0, w1, dk, db, bool(cpr), "poly" if spline is None else "bspline",
                                 *(spline or (0, 0, 0, 0)))
        assert binding.sfft_num_unknowns(cfg) == oracle.num_unknowns(oc)


def test_bspline_config_checks(lib):
    """Basis fields are checked before any CUDA call."""
    h = ctypes.c_void_p()
    for spline, dk, want in (((4, 0, 1, 0), 0, binding.SFFT_ERR_UNSUPPORTED),   # degree above 3
                             ((2, 4, 1, 0), 0, binding.SFFT_ERR_UNSUPPORTED),   # K = 7 > 6
                             ((2, 0, 1, 0), 1, binding.SFFT_ERR_INVALID),       # dk must be 0
                             ((-1, 0, 1, 0), 0, binding.SFFT_ERR_INVALID)):
        cfg = binding.make_config(64, 64, 2, 2, dk, 0, 1, spline=spline)
        assert lib.sfft_plan_create(ctypes.byref(cfg), None, ctypes.byref(h)) == want
    bad = binding.make_config(64, 64, 2, 2, 0, 0, 1)
    bad.basis = 7
    assert lib.sfft_plan_create(ctypes.byref(bad), None, ctypes.byref(h)) == binding.SFFT_ERR_INVALID


def test_set_tuning_checks_before_use(lib):
    """Out-of-range launch shapes are rejected before the plan is touched."""
    fake = ctypes.c_void_p(4096)  # never dereferenced: every call below is rejected first
    arr = lambda *v: (ctypes.c_int32 * binding.SFFT_TUNING_LEN)(*v)
    assert lib.sfft_plan_set_tuning(None, arr(0, 0, 0, 0, 0)) == binding.SFFT_ERR_INVALID
    assert lib.sfft_plan_set_tuning(fake, None) == binding.SFFT_ERR_INVALID
    for bad in ((3, 0, 0, 0, 0), (32, 0, 0, 0, 0), (-1, 0, 0, 0, 0), (0, 5, 0, 0, 0), (0, 0, -1, 0, 0),
                (0, 0, 0, 513, 0), (0, 0, 0, 0, 3), (0, 0, 0, 0, -1)):
        assert lib.sfft_plan_set_tuning(fake, arr(*bad)) == binding.SFFT_ERR_INVALID
    assert lib.sfft_plan_tuning(None, arr(0, 0, 0, 0, 0)) == binding.SFFT_ERR_INVALID


def test_solve_panel_checks_before_use(lib):
    """Only 32 and 64 are panel widths; the plan is not touched otherwise."""
    fake = ctypes.c_void_p(4096)  # never dereferenced: every call below is rejected first
    assert lib.sfft_plan_set_solve_panel(None, 32) == binding.SFFT_ERR_INVALID
    for bad in (0, 16, 48, 96, 128, -64):
        assert lib.sfft_plan_set_solve_panel(fake, bad) == binding.SFFT_ERR_INVALID
    w = ctypes.c_int32()
    assert lib.sfft_plan_solve_panel(None, ctypes.byref(w)) == binding.SFFT_ERR_INVALID
    assert lib.sfft_plan_solve_panel(fake, None) == binding.SFFT_ERR_INVALID


def test_misaligned_images_rejected(lib):
    """Images and masks must be 16-byte aligned (vector loads); checked before any use."""
    fake = ctypes.c_void_p(4096)  # never dereferenced: every call below is rejected first
    odd = ctypes.c_void_p(4096 + 4)
    ok = ctypes.c_void_p(8192)
    assert lib.sfft_build_system(fake, odd, ok, None, ok, ok, None) == binding.SFFT_ERR_INVALID
    assert lib.sfft_build_system(fake, ok, odd, None, ok, ok, None) == binding.SFFT_ERR_INVALID
    assert lib.sfft_build_system(fake, ok, ok, ctypes.c_void_p(4096 + 8), ok, ok, None) == binding.SFFT_ERR_INVALID
    assert lib.sfft_run_pair(fake, odd, ok, None, None, None, None, None, ctypes.c_void_p(12288), None) == \
        binding.SFFT_ERR_INVALID
    assert lib.sfft_subtract(fake, ok, odd, ok, ctypes.c_void_p(12288), None) == binding.SFFT_ERR_INVALID
    req = binding.make_request(odd.value, ok.value, ctypes.c_void_p(12288).value)
    t = binding.sfft_ticket()
    assert lib.sfft_submit(fake, ctypes.byref(req), ctypes.byref(t)) == binding.SFFT_ERR_INVALID


def test_header_serves_a_plain_c_program(lib, tmp_path):
    """include/sfft.h compiles as C99 with warnings as errors, and a C program
    linked against libsfft.so (no torch, no CUDA headers) calls the entry
    points that need no GPU: the unknown count of a polynomial and a B-spline
    configuration equals the oracle's, destroying a NULL plan is a no-op, and
    invalid arguments come back as status codes."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(binding.LIB)
    src = tmp_path / "use_sfft.c"
    src.write_text(r"""
#include "sfft.h"
#include <stdio.h>
#include <string.h>

static int count(int basis, int cpr, int32_t *n) {
    sfft_config c;
    memset(&c, 0, sizeof c);
    c.n0 = 4096; c.n1 = 4096; c.w0 = 8; c.w1 = 8; c.const_phot_ratio = cpr;
    c.dtype = SFFT_F32; c.precision = SFFT_PREC_MIXED; c.basis = basis;
    if (basis == SFFT_BASIS_POLY) { c.dk = 2; c.db = 2; }
    else { c.kdeg = 1; c.kint = 1; c.bdeg = 2; c.bint = 1; }
    return sfft_num_unknowns(&c, n);
}

int main(void) {
    int32_t np = 0, nb = 0;
    if (count(SFFT_BASIS_POLY, 1, &np) != SFFT_OK) return 2;
    if (count(SFFT_BASIS_BSPLINE, 0, &nb) != SFFT_OK) return 3;
    if (sfft_num_unknowns(NULL, &np) != SFFT_ERR_INVALID) return 4;
    if (sfft_plan_destroy(NULL) != SFFT_OK) return 5;          /* documented no-op */
    uint64_t bytes = 0;
    if (sfft_plan_workspace_bytes(NULL, &bytes) != SFFT_ERR_INVALID) return 6;
    printf("%d %d %s\n", (int)np, (int)nb, sfft_status_string(SFFT_ERR_SINGULAR));
    return 0;
}
""")
    exe = tmp_path / "use_sfft"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(root, "include"),
                    str(src), "-L", libdir, "-lsfft", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split(None, 2)
    poly = oracle.OracleConfig(4096, 4096, 8, 8, 2, 2, True)
    spl = oracle.OracleConfig(4096, 4096, 8, 8, 0, 0, False, "bspline", 1, 1, 2, 1)
    assert int(out[0]) == oracle.num_unknowns(poly) == 1735
    assert int(out[1]) == oracle.num_unknowns(spl)
    assert out[2].strip() == binding.status_string(-4)


def test_create_rejects_configurations_before_device_use(lib):
    """Plan, server and pool creation check their arguments before any CUDA
    call (so this runs without a GPU): sizes outside [16, 4096], lag ranges
    that do not fit one period (4w + 1 <= n, and <= 64 along a power-of-two
    x axis), degrees above 3, B-spline limits, unknown enums and NULL outputs
    each return their status, and the output handle is left NULL."""
    INV, UNS = binding.SFFT_ERR_INVALID, -8
    base = dict(n0=64, n1=64, w0=2, w1=2, dk=1, db=1, cpr=1)

    def cfg(spline=None, dtype="float32", precision="mixed", **kw):
        a = dict(base, **kw)
        return binding.make_config(a["n0"], a["n1"], a["w0"], a["w1"], a["dk"], a["db"], a["cpr"],
                                   dtype, precision, spline)

    def bad(c, field, value):
        setattr(c, field, value)
        return c

    cases = [
        (cfg(n0=15), UNS), (cfg(n1=15), UNS), (cfg(n0=4097), UNS), (cfg(n1=4097), UNS), (cfg(n0=0), UNS),
        (cfg(n0=4096, w0=16), UNS),           # 4 w0 + 1 = 65 > 64 along a power-of-two x axis
        (cfg(n0=100, n1=100, w0=25), UNS),    # 4 w0 + 1 = 101 > n0
        (cfg(n1=64, w1=16), UNS),             # 4 w1 + 1 = 65 > n1
        (cfg(w0=-1), INV), (cfg(w1=-1), INV),
        (cfg(dk=4), UNS), (cfg(db=4), UNS), (cfg(dk=-1), INV),
        (bad(cfg(), "dtype", 2), INV), (bad(cfg(), "precision", 5), INV), (bad(cfg(), "basis", 7), INV),
        (cfg(spline=(1, 1, 1, 1)), INV),                  # B-splines need dk = db = 0
        (cfg(spline=(4, 0, 1, 0), dk=0, db=0), UNS),      # degree above 3
        (cfg(spline=(3, 3, 1, 0), dk=0, db=0), UNS),      # 7 functions per axis
        (cfg(spline=(1, -1, 1, 0), dk=0, db=0), INV),
    ]
    for c, want in cases:
        h = ctypes.c_void_p(1234)
        assert lib.sfft_plan_create(ctypes.byref(c), None, ctypes.byref(h)) == want, c
        assert h.value is None
        h = ctypes.c_void_p(1234)
        assert lib.sfft_server_create(ctypes.byref(c), 2, 1, ctypes.byref(h)) == want, c
        assert h.value is None
    good = cfg()
    h = ctypes.c_void_p()
    assert lib.sfft_plan_create(None, None, ctypes.byref(h)) == INV
    assert lib.sfft_plan_create(ctypes.byref(good), None, None) == INV
    for depth, batch in [(0, 1), (9, 1), (2, 0), (2, 3)]:
        assert lib.sfft_server_create(ctypes.byref(good), depth, batch, ctypes.byref(h)) == INV
        assert lib.sfft_pool_create(ctypes.c_uint64(1 << 30), depth, batch, ctypes.byref(h)) == INV
    assert lib.sfft_pool_create(ctypes.c_uint64(0), 2, 1, ctypes.byref(h)) == INV
    assert lib.sfft_pool_create(ctypes.c_uint64(1 << 30), 2, 1, None) == INV
