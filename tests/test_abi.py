"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[ \t]*(?:const\s+)?[A-Za-z_][\w]*[\s\*]+(kf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1605_05508_gb300 import build as B
    return B.build()


def test_header_declares_the_fit_entry_points():
    names = declared_functions()
    for n in ("kf_create", "kf_destroy", "kf_fit", "kf_fit_fused", "kf_fit_f64", "kf_fit_host", "kf_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert set(declared_functions()) <= exported


def test_strerror_and_argument_checks_need_no_gpu(libpath):
    from paper_1605_05508_gb300 import kf
    lib = kf.lib()
    assert lib.kf_strerror(kf.KF_EINVAL) == b"invalid argument"
    assert lib.kf_strerror(0) == b"ok"
    # rejected before any CUDA call
    assert lib.kf_create(None, None, 0, 0) == kf.KF_EINVAL
    radii = (ctypes.c_float * 3)(4.0, 3.0, 8.0)  # not increasing
    cfg = kf.kf_config(3.8, 3, radii, 0.01, 0.1, 30.0, 6, None, 0.13957)
    h = ctypes.c_void_p()
    assert lib.kf_create(ctypes.byref(h), ctypes.byref(cfg), 0, 0) == kf.KF_EINVAL
    cfg = kf.kf_config(3.8, 3, (ctypes.c_float * 3)(4.0, 8.0, 12.0), 0.01, 0.1, 30.0, 9, None, 0.13957)  # max_cands > 8
    assert lib.kf_create(ctypes.byref(h), ctypes.byref(cfg), 0, 0) == kf.KF_EINVAL
    good = (ctypes.c_float * 3)(4.0, 8.0, 12.0)
    for x0, m in (((0.01, -0.1, 0.0), 0.14), ((0.01, 1.5, 0.0), 0.14), ((0.0, 0.0, 0.0), -1.0)):
        cfg = kf.kf_config(3.8, 3, good, 0.01, 0.1, 30.0, 6, (ctypes.c_float * 3)(*x0), m)  # bad material
        assert lib.kf_create(ctypes.byref(h), ctypes.byref(cfg), 0, 0) == kf.KF_EINVAL
    assert lib.kf_fit(None, None, None, None, None, None, None) == kf.KF_EINVAL
    # launch parameters: null context or output, and no GPU needed to reject them
    t = kf.kf_tuning(128, 0, 8, 0, 0, 0, 0)
    assert lib.kf_get_tuning(None, ctypes.byref(t)) == kf.KF_EINVAL
    assert lib.kf_set_tuning(None, ctypes.byref(t)) == kf.KF_EINVAL
    assert lib.kf_autotune_fit(None, None, None, None, None, None, None, None) == kf.KF_EINVAL
    assert lib.kf_autotune_build(None, None, None, None, 6, None, None, None) == kf.KF_EINVAL
    # measured peaks and the staged-wait test hook
    v = ctypes.c_double()
    assert lib.kf_measure_peak(None, kf.PEAK_FP32, None, ctypes.byref(v)) == kf.KF_EINVAL
    assert lib.kf_test_stage_fault(None, -1, 0) == kf.KF_EINVAL


def test_binding_constants_match_the_header():
    """Every numeric #define of include/kf.h that the binding mirrors has the
    same value there (error codes, status bits, bin grid, size limits)."""
    import re
    from paper_1605_05508_gb300 import kf
    hdr = open(os.path.join(ROOT, "include", "kf.h")).read()
    defs = {}
    for name, expr in re.findall(r"^#define (KF_\w+)\s+(.+?)\s*(?:/\*.*)?$", hdr, flags=re.M):
        e = expr.strip().rstrip("f")
        for k, v in sorted(defs.items(), key=lambda kv: -len(kv[0])):
            e = e.replace(k, repr(v))
        try:
            defs[name] = eval(e, {"__builtins__": {}})
        except Exception:
            pass
    mirror = {"KF_OK": kf.KF_OK, "KF_EINVAL": kf.KF_EINVAL, "KF_ENOMEM": kf.KF_ENOMEM, "KF_EAGAIN": kf.KF_EAGAIN,
              "KF_ETIMEDOUT": kf.KF_ETIMEDOUT, "KF_ECUDA": kf.KF_ECUDA, "KF_ENOTSUP": kf.KF_ENOTSUP,
              "KF_ST_NOT_REACHED": kf.ST_NOT_REACHED, "KF_ST_NEWTON_FAIL": kf.ST_NEWTON_FAIL,
              "KF_ST_TANGENT": kf.ST_TANGENT, "KF_ST_NOT_PD": kf.ST_NOT_PD, "KF_ST_NO_HIT": kf.ST_NO_HIT,
              "KF_ST_DEVICE_TIMEOUT": kf.ST_DEVICE_TIMEOUT, "KF_ST_STOPPED": kf.ST_STOPPED,
              "KF_BIN_ETA": kf.BIN_ETA, "KF_BIN_PHI": kf.BIN_PHI, "KF_BIN_ETA_MAX": kf.BIN_ETA_MAX,
              "KF_NBINS": kf.NBINS, "KF_BIN_PHI_FINE": kf.BIN_PHI_FINE, "KF_NBINS_FINE": kf.NBINS_FINE,
              "KF_MAX_HITS_PER_SEGMENT": kf.MAX_HITS_PER_SEGMENT,
              "KF_MAX_SLOTS": kf.MAX_SLOTS, "KF_NOALLOC_MAX_TRACKS": kf.NOALLOC_MAX_TRACKS,
              "KF_PEAK_FP32": kf.PEAK_FP32, "KF_PEAK_FP64": kf.PEAK_FP64}
    for name, value in mirror.items():
        assert name in defs, name
        assert defs[name] == value, (name, defs[name], value)


def test_binding_structures_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the
    C compiler gives the header's struct of the same name (a plain C program
    built from include/kf.h prints them)."""
    import shutil
    from paper_1605_05508_gb300 import kf
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = [getattr(kf, n) for n in ("kf_config", "kf_tracks", "kf_tracks_f64", "kf_track_hits", "kf_layer_hits",
                                        "kf_layer_hit_bins", "kf_build_result", "kf_serve_config", "kf_event",
                                        "kf_event_result", "kf_serve_stats", "kf_tuning", "kf_build_result_f64")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kf.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for f, *_ in st._fields_:
            lines.append(f'  printf("{st.__name__} {f} %zu\\n", offsetof({st.__name__}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = ln.split()
        got[(name, field)] = int(value)
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for f, *_ in st._fields_:
            assert got[(st.__name__, f)] == getattr(st, f).offset, (st.__name__, f)


def test_serve_driver_is_built_and_rejects_a_bad_pool(libpath, tmp_path):
    """The native serving driver links against libkf and refuses a file that
    is not an event pool before any CUDA call (exit status 2)."""
    from paper_1605_05508_gb300 import build as B
    assert os.path.exists(B.DRIVER)
    bad = tmp_path / "bad.kfpool"
    bad.write_bytes(b"NOPE" + b"\0" * 64)
    r = subprocess.run([B.DRIVER, str(bad), "4", "0", "1", "1"], capture_output=True, text=True)
    assert r.returncode == 2, (r.returncode, r.stderr)
    r = subprocess.run([B.DRIVER], capture_output=True, text=True)
    assert r.returncode == 2 and "usage" in r.stderr
