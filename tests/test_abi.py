"""CPU-side checks of the C-ABI library: it loads, exports every entry point that
include/mmkfvs.h declares, and its host logic (time-step rule, argument validation) matches the
oracle and the declared contract.  No GPU work is issued here."""
import ctypes
import os
import re

import pytest

from paper_2509_21832_gb300 import api
from paper_2509_21832_gb300 import inputs as I
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mm(?:1d)?_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = api.load()
    names = declared_symbols()
    assert len(names) >= 16
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(api.EXPORTS) <= names


def test_dt_rule_matches_oracle():
    cases = [I.sod_1d2v().grid, I.Grid(nx=320, ny=320, x0=-1, x1=1, y0=-1, y1=1, v1min=-9, v1max=9,
                                       v2min=-9, v2max=9),
             I.Grid(nx=256, ny=256, nv1=32, nv2=32), I.Grid(nx=17, ny=5, v1min=-3, v1max=5)]
    for g in cases:
        for form in (I.CFL_MIN, I.CFL_SUM):
            for tf in (0.0, 0.07, 0.2):
                a = api.mm_dt_for_cfl(g, 0.8, tf, form)
                b = O.dt_for_cfl(g, 0.8, tf, form)
                assert a[1] == b[1] and abs(a[0] - b[0]) <= 1e-15 * b[0]


def _create_status(grid, params):
    L = api.load()
    g, p = api.to_c_grid(grid), api.to_c_params(params)
    ctx = ctypes.c_void_p()
    return L.mm_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(ctx))


@pytest.mark.parametrize("mutate", [
    lambda g, p: setattr(p, "nu", 1.0),
    lambda g, p: setattr(p, "nu", -1.5),
    lambda g, p: setattr(p, "bc", (I.PERIODIC, I.EXTRAP, I.EXTRAP, I.EXTRAP)),
    lambda g, p: setattr(p, "bc", (I.SPECULAR,) * 4) or setattr(g, "v1min", -7.0),
    lambda g, p: setattr(g, "nx", 0),
    lambda g, p: setattr(g, "nv1", 0),
    lambda g, p: setattr(g, "nv2", 2000),
    lambda g, p: setattr(p, "precision", 7),
    lambda g, p: setattr(p, "tau0", 0.0),
    lambda g, p: setattr(p, "bc", (I.DIFFUSE,) * 4) or setattr(p, "wall_T", (1.0, 0.0, 1.0, 1.0)),
    lambda g, p: setattr(g, "x1", g.x0),
])
def test_create_rejects_invalid_arguments_before_device_work(mutate):
    g = I.Grid(nx=4, ny=4, nv1=8, nv2=8)
    p = I.Params()
    mutate(g, p)
    assert _create_status(g, p) == api.MM_ERR_INVALID_ARG


def test_device_bytes():
    g = I.Grid(nx=256, ny=256, nv1=32, nv2=32)
    p = I.Params(bc=(I.SPECULAR,) * 4)
    b = api.mm_device_bytes(g, p)
    assert b >= 2 * g.nphase * 8
    p.precision = I.PREC_G_FP32
    assert api.mm_device_bytes(g, p) < b


def test_header_is_plain_c():
    """include/mmkfvs.h compiles as C99 (pedantic) and as C++: a C ABI usable from both."""
    import shutil
    import subprocess
    import tempfile
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    inc = os.path.join(ROOT, "include")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "use.c")
        with open(src, "w") as f:
            f.write('#include "mmkfvs.h"\nint main(void) { mm_grid g; (void)g; return 0; }\n')
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                               "-fsyntax-only", "-I" + inc, src])
        if shutil.which("g++"):
            subprocess.check_call(["g++", "-x", "c++", "-std=c++17", "-Wall", "-Werror",
                                   "-fsyntax-only", "-I" + inc, src])


def test_scratch_bytes_bookkeeping():
    """mm_device_bytes = g + Q + mm_scratch_bytes; every scratch piece is rounded to 256 bytes; an
    invalid problem needs 0."""
    for g, p, gsz in [(I.Grid(nx=20, ny=12, nv1=32, nv2=32), I.Params(bc=(I.SPECULAR,) * 4), 8),
                      (I.Grid(nx=9, ny=18, nv1=24, nv2=24),
                       I.Params(bc=(I.EXTRAP, I.EXTRAP, I.DIFFUSE, I.EXTRAP),
                                precision=I.PREC_G_FP32), 4)]:
        nc = g.nx * g.ny
        s = api.mm_scratch_bytes(g, p)
        assert s > 0 and s % 256 == 0
        assert api.mm_device_bytes(g, p) == nc * g.nv1 * g.nv2 * gsz + 6 * nc * 8 + s
        # at least the split-step copy of g, the heat flux and the per-cell coefficients
        assert s >= nc * g.nv1 * g.nv2 * gsz + 4 * nc * 8
    bad = I.Grid(nx=0, ny=4)
    assert api.mm_scratch_bytes(bad, I.Params()) == 0


def test_create_borrowed_rejects_bad_buffers_without_gpu_work():
    """Argument checks of mm_create_borrowed come before any device call: NULL pointers,
    misalignment and too little scratch are MM_ERR_INVALID_ARG."""
    g, p = I.Grid(nx=8, ny=8, nv1=16, nv2=16), I.Params()
    need = api.mm_scratch_bytes(g, p)
    base = 1 << 20  # never dereferenced: every case fails its checks first
    cases = [(0, base, base, need), (base, 0, base, need), (base, base, 0, need),
             (base + 8, base, base, need), (base, base + 8, base, need),
             (base, base, base + 128, need), (base, base, base, need - 1)]
    for q, gg, sc, nb in cases:
        st, _ = api.mm_create_borrowed(g, p, q, gg, sc, nb)
        assert st == api.MM_ERR_INVALID_ARG, (q, gg, sc, nb)
    st, _ = api.mm_create_borrowed(I.Grid(nx=0, ny=8), p, base, base, base, need)
    assert st == api.MM_ERR_INVALID_ARG


def test_fp32_g_meshes_beyond_shared_memory_are_rejected():
    """FP32 g keeps three rows of G* per warp in shared memory: velocity meshes whose kernel would
    need more than the 227 KB a CTA can have are rejected when the problem is validated (before
    any device work), the others accepted."""
    p32 = I.Params(precision=I.PREC_G_FP32, bc=(I.PERIODIC,) * 4)
    assert api.mm_device_bytes(I.Grid(nx=8, ny=8, nv1=32, nv2=100), p32) > 0
    assert api.mm_device_bytes(I.Grid(nx=8, ny=8, nv1=32, nv2=128), p32) == 0
    assert api.mm_device_bytes(I.Grid(nx=8, ny=8, nv1=32, nv2=1024), p32) == 0
    # the FP64 kernels fit at every accepted mesh
    assert api.mm_device_bytes(I.Grid(nx=8, ny=8, nv1=32, nv2=1024), I.Params()) > 0


def test_missing_library_fails_loudly():
    """Without the built library the binding raises instead of computing anything on the CPU."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); "
            "from paper_2509_21832_gb300 import build as b, api; "
            "b.LIB = '/nonexistent/libmmkfvs.so'; api._lib = None\n"
            "try:\n    api.load(build_if_needed=False)\n    print('loaded')\n"
            "except ImportError as e:\n    print('ImportError', e)" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.stdout.startswith("ImportError"), r.stdout + r.stderr


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it."""
    import ast
    pkg = os.path.join(ROOT, "paper_2509_21832_gb300")
    for fn in sorted(os.listdir(pkg)):
        if not fn.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, fn)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (fn, mods)
