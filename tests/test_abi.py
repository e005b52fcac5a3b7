"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry
point include/pond.h declares, and its host-side validation works without a
GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1806_05089_gb300 import pond

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "pond.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(pond_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    lib = pond.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pond.EXPORTS)


def test_version_and_defaults():
    assert "D2Q16" in pond.pond_version() and "D2Q9" in pond.pond_version()
    c64 = pond.pond_config_default(pond.POND_FP64)
    assert (c64.eps_abs, c64.eps_rel) == (1e-12, 1e-10)  # App. E
    assert c64.max_iter == 20 and c64.thermal == 1 and c64.dt == 1.0
    assert c64.lattice == pond.POND_D2Q16
    c32 = pond.pond_config_default(pond.POND_FP32_MIXED)
    assert c32.precision == pond.POND_FP32_MIXED and c32.eps_rel >= 1e-7


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    cfg = pond.pond_config_default(pond.POND_FP64)
    lib = pond.load()
    out = ctypes.c_void_p()
    nx = (ctypes.c_int32 * 1)(8)
    ny = (ctypes.c_int32 * 1)(0)
    assert lib.pond_create(ctypes.byref(cfg), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    ny[0] = 8
    assert lib.pond_create(ctypes.byref(cfg), 0, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    bad = pond.pond_config_default(pond.POND_FP64)
    bad.nu = -1.0
    assert lib.pond_create(ctypes.byref(bad), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    # the direct FP64 kernels step one grid; FP64 ensembles run staged
    nx2 = (ctypes.c_int32 * 2)(8, 8)
    ny2 = (ctypes.c_int32 * 2)(8, 8)
    direct = pond.pond_config_default(pond.POND_FP64)
    direct.kernel = pond.POND_KERNEL_DIRECT
    assert lib.pond_create(ctypes.byref(direct), 2, nx2, ny2, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    direct.kernel = pond.POND_KERNEL_DEFAULT
    direct.nodes_per_warp = 2  # a direct-only mapping
    assert lib.pond_create(ctypes.byref(direct), 2, nx2, ny2, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    assert lib.pond_step(None, 1, None) == pond.POND_ERR_ARG
    assert lib.pond_last_error(None) == b"no context"
    # lattice: D2Q16 or D2Q9 only; the paired tile shape is D2Q16-only
    bad = pond.pond_config_default(pond.POND_FP32_MIXED)
    bad.lattice = 2
    assert lib.pond_create(ctypes.byref(bad), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    bad.lattice = pond.POND_D2Q9
    bad.tile_rows = -16
    assert lib.pond_create(ctypes.byref(bad), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    # three nodes per warp is a D2Q9 mapping
    bad = pond.pond_config_default(pond.POND_FP64)
    bad.nodes_per_warp = 3
    assert lib.pond_create(ctypes.byref(bad), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    bad.lattice = pond.POND_D2Q9
    for npw in (-1, 4, 16, 31, 33):
        bad.nodes_per_warp = npw
        assert lib.pond_create(ctypes.byref(bad), 1, nx, ny, None, ctypes.byref(out)) == pond.POND_ERR_ARG
    # one node per thread (32) passes the argument check on both lattices;
    # without a GPU the call then fails on the device, not on its arguments
    for lattice in (pond.POND_D2Q16, pond.POND_D2Q9):
        ok = pond.pond_config_default(pond.POND_FP64)
        ok.lattice = lattice
        ok.nodes_per_warp = 32
        st = lib.pond_create(ctypes.byref(ok), 1, nx, ny, None, ctypes.byref(out))
        assert st != pond.POND_ERR_ARG
        if st == pond.POND_OK:
            lib.pond_destroy(out)


def test_no_cpu_fallback_without_gpu():
    """Without a GPU the library reports a CUDA error instead of computing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = pond.pond_config_default(pond.POND_FP64)
    with pytest.raises(pond.PondError) as e:
        pond.pond_create(cfg, [8], [8])
    assert e.value.status in (pond.POND_ERR_CUDA, pond.POND_ERR_OOM)


def test_header_is_plain_c_and_structs_match_the_binding(tmp_path):
    """include/pond.h compiles as C99 (-Wall -Wextra -pedantic -Werror), and
    the sizes and field offsets of pond_config and pond_stats seen by a C
    compiler equal those of the ctypes structures of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pond.h"', 'int main(void) {']
    for cname, pyst in (("pond_config", pond.pond_config), ("pond_stats", pond.pond_stats)):
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in pyst._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ['  return 0;', '}']
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = {}
    for line in out:
        p = line.split()
        if len(p) == 3:
            seen[(p[0], p[1])] = int(p[2])
    for cname, pyst in (("pond_config", pond.pond_config), ("pond_stats", pond.pond_stats)):
        assert seen[(cname, "size")] == ctypes.sizeof(pyst), cname
        for field, _ in pyst._fields_:
            assert seen[(cname, field)] == getattr(pyst, field).offset, (cname, field)


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    """A C99 program links against libpond.so by its exported names and calls
    the argument checks of the boundary: the version string, the defaults,
    rejections of bad arguments and, without a GPU, a CUDA status from a
    valid pond_create (no CPU fallback)."""
    import shutil
    import subprocess
    import torch
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pond.load()
    libdir = os.path.dirname(pond._build.LIB)
    src = tmp_path / "client.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "pond.h"

int main(int argc, char** argv) {
    int have_gpu = argc > 1 && strcmp(argv[1], "gpu") == 0;
    pond_config cfg;
    pond_config_default(&cfg, POND_FP64);
    if (cfg.precision != POND_FP64 || !(cfg.nu > 0.0)) return 10;
    if (strstr(pond_version(), "D2Q9") == NULL) return 11;
    int32_t nx = 8, ny = 0;
    pond_ctx* ctx = NULL;
    if (pond_create(&cfg, 1, &nx, &ny, NULL, &ctx) != POND_ERR_ARG) return 12;
    ny = 8;
    cfg.nu = -1.0;
    if (pond_create(&cfg, 1, &nx, &ny, NULL, &ctx) != POND_ERR_ARG) return 13;
    pond_config_default(&cfg, POND_FP64);
    cfg.nodes_per_warp = 5;
    if (pond_create(&cfg, 1, &nx, &ny, NULL, &ctx) != POND_ERR_ARG) return 14;
    if (pond_step(NULL, 1, NULL) != POND_ERR_ARG) return 15;
    if (strcmp(pond_last_error(NULL), "no context") != 0) return 16;
    pond_config_default(&cfg, POND_FP64);
    pond_status st = pond_create(&cfg, 1, &nx, &ny, NULL, &ctx);
    if (have_gpu) {
        if (st != POND_OK) return 17;
        pond_destroy(ctx);
    } else if (st != POND_ERR_CUDA && st != POND_ERR_OOM) {
        return 18;
    }
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "client"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lpond", "-Wl,-rpath," + libdir], check=True)
    args = [str(exe)] + (["gpu"] if torch.cuda.is_available() else [])
    r = subprocess.run(args, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def _ctype_of(decl: str):
    """ctypes type of one C parameter or return type of include/pond.h."""
    t = " ".join(decl.replace("const", " ").split())
    pointers = t.count("*")
    base = t.replace("*", "").strip()
    if pointers == 0:
        return {"int32_t": ctypes.c_int32, "double": ctypes.c_double,
                "pond_status": ctypes.c_int32, "void": None}[base]
    if pointers == 2:
        assert base == "pond_ctx", decl
        return ctypes.POINTER(ctypes.c_void_p)
    if base == "char":
        return ctypes.c_char_p
    return {"pond_ctx": ctypes.c_void_p, "void": ctypes.c_void_p,
            "pond_config": ctypes.POINTER(pond.pond_config),
            "pond_stats": ctypes.POINTER(pond.pond_stats),
            "int32_t": ctypes.POINTER(ctypes.c_int32),
            "double": ctypes.POINTER(ctypes.c_double)}[base]


def test_binding_signatures_match_the_header():
    """Every prototype of include/pond.h against the ctypes argtypes and
    restype the binding declares: the same number of parameters, each of the
    matching ctypes type (a mismatch would pass pointers or sizes in the
    wrong slots, which no CPU test would otherwise see)."""
    hdr = open(os.path.join(ROOT, "include", "pond.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    protos = re.findall(r"(pond_status|void|const\s+char\s*\*)\s*\b(pond_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                        hdr)
    assert {name for _, name, _ in protos} == set(pond.EXPORTS)
    lib = pond.load()
    for ret, name, params in protos:
        fn = getattr(lib, name)
        want_ret = _ctype_of(ret)
        assert fn.restype == want_ret, (name, fn.restype, want_ret)
        decls = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        # drop each parameter's name: the last identifier of the declaration
        types = [re.sub(r"\b[A-Za-z_][A-Za-z0-9_]*\s*$", "", d) for d in decls]
        assert len(fn.argtypes) == len(types), (name, fn.argtypes, types)
        for i, (have, t) in enumerate(zip(fn.argtypes, types)):
            want = _ctype_of(t)
            if "*" not in t:                       # scalars: the exact type
                assert have == want, (name, i, have, want)
            elif have is not ctypes.c_void_p:      # a typed pointer: the same pointee
                assert issubclass(have, ctypes._Pointer) and issubclass(want, ctypes._Pointer), \
                    (name, i, have, want)
                assert have._type_ is want._type_, (name, i, have, want)


def test_every_context_call_refuses_a_null_context():
    """Each entry point that takes a pond_ctx returns POND_ERR_ARG for a NULL
    context (with NULL or zero for every other argument) before it touches
    anything: no crash, no CUDA call, the same on a machine without a GPU."""
    lib = pond.load()
    d = ctypes.c_double(0.0)
    calls = {
        "pond_set_stream": (None, None),
        "pond_set_state": (None, 0, None, None, None, None, None, 0),
        "pond_step": (None, 1, None),
        "pond_moments": (None, 0, None, None, None, None, 0),
        "pond_get_state": (None, 0, None, None, None, None, 0),
        "pond_iterations": (None, 0, None, 0),
        "pond_adjoint_step": (None, None, None, None, None, None),
        "pond_adjoint_step_given": (None, None, None, None, None, None, None, None, None),
        "pond_adjoint_nu_bar": (None, ctypes.byref(d)),
        "pond_adjoint_init": (None, None, None),
        "pond_set_interior": (None, 0, 0, 0, 1, 1),
        "pond_pack_rect": (None, 0, 0, 0, 1, 1, None),
        "pond_unpack_rect": (None, 0, 0, 0, 1, 1, None),
        "pond_max_displacement": (None, 0, ctypes.byref(d)),
    }
    hdr = open(os.path.join(ROOT, "include", "pond.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    takes_ctx = set(re.findall(r"pond_status\s+(pond_[a-z0-9_]+)\s*\(\s*(?:const\s+)?pond_ctx\s*\*", hdr))
    assert takes_ctx == set(calls)
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == pond.POND_ERR_ARG, name
    lib.pond_destroy(None)
    assert lib.pond_last_error(None) == b"no context"


def test_context_free_calls_check_their_arguments_first():
    """pond_step_fp64_noalloc and pond_measure_peak refuse bad arguments with
    POND_ERR_ARG before any CUDA call (so without a GPU as well).  Without a
    GPU a valid call ends at the device lookup with POND_ERR_CUDA and never
    uses its pointers (no CPU fallback)."""
    import torch
    lib = pond.load()
    cfg = pond.pond_config_default(pond.POND_FP64)
    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)          # never dereferenced: the checks fail first
    arrays = [p] * 8

    def noalloc(c, nx, ny, arrs):
        return lib.pond_step_fp64_noalloc(ctypes.byref(c) if c is not None else None, nx, ny,
                                          *arrs, None, None, None)

    assert noalloc(None, 1, 1, arrays) == pond.POND_ERR_ARG
    for i in range(8):
        holed = list(arrays)
        holed[i] = None
        assert noalloc(cfg, 1, 1, holed) == pond.POND_ERR_ARG, i
    for nx, ny in ((0, 4), (4, 0), (-1, 4), (513, 512)):  # 262656 > POND_NOALLOC_MAX_NODES
        assert noalloc(cfg, nx, ny, arrays) == pond.POND_ERR_ARG, (nx, ny)
    mixed = pond.pond_config_default(pond.POND_FP32_MIXED)
    assert noalloc(mixed, 1, 1, arrays) == pond.POND_ERR_ARG
    bad = pond.pond_config_default(pond.POND_FP64)
    bad.lattice = 7
    assert noalloc(bad, 1, 1, arrays) == pond.POND_ERR_ARG
    if not torch.cuda.is_available():
        assert noalloc(cfg, 1, 1, arrays) == pond.POND_ERR_CUDA
        assert noalloc(cfg, 512, 512, arrays) == pond.POND_ERR_CUDA   # the largest grid passes

    tf = ctypes.c_double(0.0)
    peak = lib.pond_measure_peak
    assert peak(pond.POND_PIPE_FP64, 1, p, None, None, None) == pond.POND_ERR_ARG
    assert peak(pond.POND_PIPE_FP64, 1, None, None, ctypes.byref(tf), None) == pond.POND_ERR_ARG
    assert peak(pond.POND_PIPE_FP64, 0, p, None, ctypes.byref(tf), None) == pond.POND_ERR_ARG
    assert peak(3, 1, p, None, ctypes.byref(tf), None) == pond.POND_ERR_ARG
    assert peak(-1, 1, p, None, ctypes.byref(tf), None) == pond.POND_ERR_ARG
