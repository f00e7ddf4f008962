"""The C-ABI library builds here, loads, and exports every symbol include/hm.h declares.

CPU only: no compute call is made (there is no GPU in this container).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_]+)\s*\(", text)) - {"hm_apply_fn"})


def test_library_builds_and_exports_all_declared_symbols():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 11
    for s in syms:
        assert hasattr(lib, s), f"libhm.so does not export {s}"
    import paper_2205_03406_gb300 as hm
    assert sorted(hm.EXPORTED) == syms


def test_binding_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives."""
    import subprocess
    import paper_2205_03406_gb300 as hm
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "hm.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(hm_config), sizeof(hm_op),'
        ' sizeof(hm_info), offsetof(hm_config, seed), offsetof(hm_op, user), offsetof(hm_info, seconds_total),'
        ' offsetof(hm_info, pool_peak_bytes), sizeof(hm_job_desc), offsetof(hm_job_desc, rank),'
        ' sizeof(hm_job_stats), sizeof(hm_server_info), offsetof(hm_server_info, apply_p99_s)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(hm.hm_config), ctypes.sizeof(hm.hm_op), ctypes.sizeof(hm.hm_info),
            hm.hm_config.seed.offset, hm.hm_op.user.offset, hm.hm_info.seconds_total.offset,
            hm.hm_info.pool_peak_bytes.offset, ctypes.sizeof(hm.hm_job_desc), hm.hm_job_desc.rank.offset,
            ctypes.sizeof(hm.hm_job_stats), ctypes.sizeof(hm.hm_server_info), hm.hm_server_info.apply_p99_s.offset]
    assert got == want


def test_binding_constants_match_header(tmp_path):
    """Formats and export selectors of the binding equal the header's."""
    import subprocess
    import paper_2205_03406_gb300 as hm
    names = ["HM_FORMAT_H1", "HM_FORMAT_UNIFORM_H1", "HM_FORMAT_H2", "HM_X_LEAF_D", "HM_X_BOX_DEGREE",
             "HM_X_H2_RANKS", "HM_X_H2_SIGMA", "HM_MIXED_BF16X6", "HM_MIXED_BF16X6_F32"]
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "hm.h"\nint main(void){'
                   + "".join(f'printf("%d\\n", (int){n});' for n in names) + 'return 0;}\n')
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [getattr(hm, n) for n in names]


def test_create_rejects_bad_configs_without_gpu():
    """Argument checks happen before any CUDA work."""
    import paper_2205_03406_gb300 as hm
    bad = [hm.Settings(d=4), hm.Settings(d=3, r=0, rank=1), hm.Settings(d=3, r=65, rank=1),
           hm.Settings(d=3, rank=-1), hm.Settings(d=3, tol=-1e-6), hm.Settings(d=3, tol=float("nan")),
           hm.Settings(d=3, r=8, rank=9), hm.Settings(d=3, rank=4, precision=7),
           hm.Settings(d=3, r=8, oversample=8, tol=1e-6), hm.Settings(d=3, leaf_size=-1, rank=4)]
    for s in bad:
        with pytest.raises(hm.HMError) as ei:
            hm.hm_create(s.to_c())
        assert ei.value.status == hm.HM_EINVAL
    with pytest.raises(hm.HMError) as ei:  # an H^2 operator keeps no per-level samples
        hm.hm_create(hm.Settings(d=3, rank=4, format=hm.HM_FORMAT_H2, keep_samples=True).to_c())
    assert ei.value.status == hm.HM_ENOTSUP
    with pytest.raises(hm.HMError) as ei:
        hm.hm_create(hm.Settings(d=3, rank=4, format=3).to_c())
    assert ei.value.status == hm.HM_EINVAL
    assert hm.hm_destroy(None) == hm.HM_OK


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2205_03406_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracle's", ""), f


def test_call_order_and_argument_checks_without_gpu():
    """The C ABI's state machine and argument checks (no device work is done
    before they pass): out-of-order calls return HM_ESTATE, null pointers and
    bad sizes HM_EINVAL, and the context stays destroyable."""
    import ctypes

    import paper_2205_03406_gb300 as hm
    L = hm.lib()
    assert L.hm_color(None, 2, None) == hm.HM_EINVAL
    assert L.hm_destroy(None) == hm.HM_OK
    for prec in (hm.HM_FP64, hm.HM_MIXED_BF16X6, hm.HM_MIXED_BF16X6_F32):
        ctx = hm.hm_create(hm.Settings(d=3, leaf_size=16, r=8, rank=4, oversample=4, precision=prec).to_c())
        try:
            nc = ctypes.c_int(0)
            op = hm.kernel_op(hm.HM_K_LAPLACE3D)
            e = ctypes.c_double(0.0)
            size = ctypes.c_size_t(0)
            info = hm.hm_info()
            # nothing is built yet
            assert L.hm_color(ctx, 2, ctypes.byref(nc)) == hm.HM_ESTATE
            assert L.hm_sample(ctx, ctypes.byref(op), 2) == hm.HM_ESTATE
            assert L.hm_compress(ctx, ctypes.byref(op), 0.0, 0) == hm.HM_ESTATE
            assert L.hm_apply(ctx, ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 0) == hm.HM_ESTATE
            assert L.hm_apply_noalloc(ctx, ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 0) == hm.HM_ESTATE
            assert L.hm_relerr(ctx, ctypes.byref(op), 20, ctypes.byref(e)) == hm.HM_ESTATE
            assert L.hm_export(ctx, hm.HM_X_PERM, 0, None, ctypes.byref(size)) == hm.HM_ESTATE
            assert L.hm_get_info(ctx, ctypes.byref(info)) == hm.HM_OK
            # null pointers and bad sizes
            assert L.hm_tree_build(ctx, None, 10, 0) == hm.HM_EINVAL
            assert "tree_build" in L.hm_last_error(ctx).decode()
            assert L.hm_tree_build(ctx, ctypes.c_void_p(16), 0, 0) == hm.HM_EINVAL
            assert L.hm_tree_build(ctx, ctypes.c_void_p(16), 10, -1) == hm.HM_EINVAL
            assert L.hm_sample(ctx, None, 2) == hm.HM_EINVAL
            assert L.hm_compress(ctx, None, 0.0, 0) == hm.HM_EINVAL
            # truncation arguments of hm_compress (checked before the call order)
            for tol, rank in ((-1.0, 0), (float("nan"), 0), (0.0, -1), (0.0, 9), (1e-6, 9)):
                assert L.hm_compress(ctx, ctypes.byref(op), tol, rank) == hm.HM_EINVAL, (tol, rank)
            for tol, rank in ((1e-6, 0), (1e-6, 3), (0.0, 8)):
                assert L.hm_compress(ctx, ctypes.byref(op), tol, rank) == hm.HM_ESTATE, (tol, rank)
            assert L.hm_get_info(ctx, None) == hm.HM_EINVAL
        finally:
            assert L.hm_destroy(ctx) == hm.HM_OK


def test_injected_allocation_failure_without_gpu(tmp_path):
    """Host-side fault injection (HM_FAULT_ALLOC_AFTER): the first device
    allocation of hm_tree_build fails with HM_ENOMEM before any CUDA call, the
    error message says so, and the context is still destroyable."""
    import subprocess
    import sys
    script = tmp_path / "inject.py"
    script.write_text(
        "import sys, ctypes\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import paper_2205_03406_gb300 as hm\n"
        "L = hm.lib()\n"
        "ctx = hm.hm_create(hm.Settings(d=3, leaf_size=16, r=8, rank=4).to_c())\n"
        "st = L.hm_tree_build(ctx, ctypes.c_void_p(16), 10, 0)\n"
        "msg = L.hm_last_error(ctx).decode()\n"
        "assert st == hm.HM_ENOMEM, st\n"
        "assert 'injected' in msg, msg\n"
        "assert L.hm_destroy(ctx) == hm.HM_OK\n"
        "print('ok')\n")
    env = dict(os.environ, HM_FAULT_ALLOC_AFTER="0")
    out = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "ok" in out.stdout, out.stdout + out.stderr


def test_server_argument_checks_without_gpu():
    """The serving entry points check their arguments before any CUDA work; with
    no device visible hm_server_create reports HM_ECUDA."""
    import ctypes

    import paper_2205_03406_gb300 as hm
    L = hm.lib()
    h = ctypes.c_void_p()
    assert L.hm_server_create(None, None) == hm.HM_EINVAL
    assert L.hm_server_create(ctypes.byref(h), ctypes.byref(hm.hm_server_config(0, 0))) == hm.HM_EINVAL
    assert L.hm_server_create(ctypes.byref(h), ctypes.byref(hm.hm_server_config(0, 65))) == hm.HM_EINVAL
    assert L.hm_server_create(ctypes.byref(h), ctypes.byref(hm.hm_server_config(0, 2))) == hm.HM_ECUDA
    assert L.hm_server_submit(None, None, None) == hm.HM_EINVAL
    assert L.hm_server_wait(None, 1, 0.0, None) == hm.HM_EINVAL
    assert L.hm_server_apply(None, 1, None, None, 1, 0) == hm.HM_EINVAL
    assert L.hm_server_release(None, 1) == hm.HM_EINVAL
    assert L.hm_server_get_info(None, None) == hm.HM_EINVAL
    assert L.hm_server_destroy(None) == hm.HM_OK
