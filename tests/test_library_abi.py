"""The C-ABI library builds, loads without a GPU and exports what include/ba.h declares."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ba.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2608_14266_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(built):
    names = built.declared_symbols(HEADER)
    assert len(names) >= 15
    out = subprocess.check_output(["nm", "-D", "--defined-only", built.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = built.lib()
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layouts_match_header(built, tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ba.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(ba_config), sizeof(ba_stats),'
                   ' offsetof(ba_config, cuda_stream), offsetof(ba_stats, iters));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    c_sizes = list(map(int, subprocess.check_output([str(exe)], text=True).split()))
    py = [ctypes.sizeof(built.BaConfig), ctypes.sizeof(built.BaStats), built.BaConfig.cuda_stream.offset,
          built.BaStats.iters.offset]
    assert c_sizes == py


def test_defaults_and_status_strings_without_gpu(built):
    import paper_2608_14266_gb300 as mm
    cfg = mm.ba_config_default()
    assert cfg.precision == mm.BA_FP64 and cfg.max_iters == 200 and cfg.mu0 == 1e-4
    assert cfg.rel_tol == 1e-8 and cfg.fixed_scan == 0 and cfg.max_consec_reject == 10
    lib = built.lib()
    assert lib.ba_status_string(1) == b"BA_ERR_INVALID_ARG"
    assert lib.ba_status_string(6) == b"BA_ERR_TIMEOUT"


def test_create_rejects_bad_config_before_touching_a_device(built):
    import paper_2608_14266_gb300 as mm
    for bad in ({"precision": 7}, {"mu0": -1.0}, {"hessian_mode": 5}, {"max_consec_reject": 0}):
        with pytest.raises(mm.BAError) as ei:
            mm.ba_create(mm.ba_config_default(**bad))
        assert ei.value.status == 1


def test_null_handle_calls_fail_cleanly(built):
    lib = built.lib()
    assert lib.ba_iterate(None, 1, None) == 1
    assert lib.ba_poses(None, None, 0) == 1
    assert lib.ba_kernel_launches(None) == 0
    lib.ba_destroy(None)


def test_product_path_has_no_cpu_fallback(built, monkeypatch):
    """With the shared library missing, the binding raises instead of computing."""
    from paper_2608_14266_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "does_not_exist.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()


def test_package_does_not_import_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_2608_14266_gb300, scenegen; "
            "assert 'oracle' not in sys.modules, 'product imported the oracle'") % ROOT
    subprocess.check_call([sys.executable, "-c", code])


def test_memory_estimate_is_host_only_and_grows_with_the_problem(built):
    """ba_estimate_bytes (the server's admission figure) needs no device: it
    grows with each size, linearly in the clusters, and its load peak includes
    what a mixed load from host memory adds per cluster: the slot staging (48
    bytes), the scan-major positions grouped by chunk (4) and that grouping's
    sort keys, buffers and scratch (14)."""
    import paper_2608_14266_gb300 as mm
    for prec in (mm.BA_FP64, mm.BA_MIXED):
        k0, p0 = mm.ba_estimate_bytes(prec, 100, 10_000, 200_000)
        assert k0 > 0 and p0 > 0
        for args in ((200, 10_000, 200_000), (100, 20_000, 200_000), (100, 10_000, 400_000)):
            k, p = mm.ba_estimate_bytes(prec, *args)
            assert k > k0 and p >= p0
        k2, _ = mm.ba_estimate_bytes(prec, 100, 10_000, 400_000)
        k4, _ = mm.ba_estimate_bytes(prec, 100, 10_000, 800_000)
        assert abs((k4 - k2) - 2 * (k2 - k0)) <= 1024  # linear in the clusters (200k, 400k, 800k)
    _, p64 = mm.ba_estimate_bytes(mm.BA_FP64, 100, 10_000, 200_000)
    _, pmx = mm.ba_estimate_bytes(mm.BA_MIXED, 100, 10_000, 200_000)
    assert pmx - p64 == (48 + 4 + 14) * 200_000
