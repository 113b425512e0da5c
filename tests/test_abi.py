"""The C-ABI library builds for sm_103a, loads, and exports every function
include/hp.h declares; argument validation happens before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2004_04334_gb300 import build, hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hp.load()


def test_header_declares_binding_exports():
    assert sorted(hp.EXPORTS) == _declared()


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a_only():
    # one -gencode, for sm_103a (checked on the build command, not the binary)
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _declared_arity():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(hp_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    arity = _declared_arity()
    assert set(arity) == set(hp.EXPORTS)
    for name, n in arity.items():
        assert len(getattr(lib, name).argtypes) == n, name


def test_status_strings(lib):
    for st in range(10):
        assert hp.status_string(st).startswith("HP_")


def _cfg(**kw):
    gain = np.full(4, 70, np.int32)
    ped = np.full(4, 100, np.int32)
    base = dict(device=0, n_modules=4, rows=160, cols=416, pixel_thr=1000, cluster_thr=4000,
                gain=gain.ctypes.data, pedestal=ped.ctypes.data, device_budget_bytes=0, max_inflight=0,
                n_streams=0, flags=0)
    base.update(kw)
    return hp.Config(**base), (gain, ped)


@pytest.mark.parametrize("bad", [dict(n_modules=0), dict(rows=0), dict(rows=257), dict(cols=513),
                                 dict(pixel_thr=0), dict(gain=None), dict(rows=256, cols=512 + 1)])
def test_create_rejects_invalid_config_without_cuda(lib, bad):
    cfg, keep = _cfg(**bad)
    h = ctypes.c_void_p()
    assert lib.hp_create(ctypes.byref(cfg), ctypes.byref(h)) == hp.HP_EINVAL
    assert not h.value


def test_create_rejects_out_of_domain_calibration(lib):
    gain = np.array([70, 127, 70, 70], np.int32)  # 255 * 127 > INT32_MAX / 66560
    ped = np.zeros(4, np.int32)
    cfg, _ = _cfg(gain=gain.ctypes.data, pedestal=ped.ctypes.data)
    h = ctypes.c_void_p()
    assert lib.hp_create(ctypes.byref(cfg), ctypes.byref(h)) == hp.HP_EINVAL


def test_null_arguments(lib):
    assert lib.hp_destroy(None) == hp.HP_EINVAL
    assert lib.hp_enqueue_event(None, None, None, 0, 0, 0, None) == hp.HP_EINVAL
    assert lib.hp_release_event(None) == hp.HP_EINVAL
    assert lib.hp_event_query(None) == hp.HP_EINVAL
    assert lib.hp_get_stats(None, None) == hp.HP_EINVAL


def test_header_is_plain_c():
    # the boundary is a C ABI: the header must compile as C on its own
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    r = subprocess.run([gcc, "-fsyntax-only", "-std=c11", "-x", "c", os.path.join(ROOT, "include", "hp.h")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


# Structures the binding mirrors: (C type in include/hp.h, binding class or
# numpy record).
_MIRRORS = [("hp_config", "Config"), ("hp_clusters", "ClustersView"), ("hp_device_clusters", "DeviceClusters"),
            ("hp_stats", "Stats"), ("hp_tuning", "Tuning"), ("hp_provenance", "Provenance"), ("hp_hits", "HitsView"),
            ("hp_serve_config", "ServeConfig"), ("hp_serve_trace_record", "TRACE_DTYPE")]


def _binding_layout(name):
    m = getattr(hp, name)
    if isinstance(m, np.dtype):
        return m.itemsize, [(f, m.fields[f][1]) for f in m.names]
    return ctypes.sizeof(m), [(f, getattr(m, f).offset) for f, _ in m._fields_]


def test_binding_structures_match_the_header_layout(tmp_path):
    """Every structure the binding mirrors has the header's size and field
    offsets, as the host C compiler lays them out (field names must match)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hp.h"', "int main(void) {"]
    for ctype, name in _MIRRORS:
        _, fields = _binding_layout(name)
        lines.append(f'printf("{name} size %zu\\n", sizeof({ctype}));')
        for f, _ in fields:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({ctype}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for _, name in _MIRRORS:
        size, fields = _binding_layout(name)
        assert got[(name, "size")] == size, name
        for f, off in fields:
            assert got[(name, f)] == off, (name, f)


def test_hash_store_capacity_formula_matches_the_kernel_header(tmp_path):
    """The GPU tests place items at the hash store's capacity with a Python
    copy of the formula; it must agree with hash_capacity in the kernels'
    header for every tile, block count and group size the tuner offers."""
    import shutil
    import subprocess

    from tests.test_gpu_hash_store import _capacity

    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(shutil.which("nvcc") or "/x/x"))),
                            "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    cases = [(t, b, it) for b, tiles in ((1, (4096, 10240)), (2, (2048, 4096)), (3, (1536, 2304, 2560)))
             for t in tiles for it in (128, 256, 512)]
    body = "\n".join(f'printf("%u\\n", hp::hash_capacity(hp::cc_smem_bytes(160, 416, {t}), {t}, {it}, '
                     f'hp::cc_digis_per_thread({b})));' for t, b, it in cases)
    src = tmp_path / "cap.cpp"
    src.write_text('#include <cstdio>\n#include "hp_internal.h"\nint main() {\n' + body + "\nreturn 0; }\n")
    exe = tmp_path / "cap"
    subprocess.run([cxx, "-std=c++17", "-I", os.path.join(ROOT, "paper_2004_04334_gb300", "csrc"), "-I", cuda_inc,
                    str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [_capacity({"tile_slots": t, "blocks_per_sm": b, "item_threads": it}) for t, b, it in cases]
    assert got == want
