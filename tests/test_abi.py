"""CPU checks of the C-ABI library: it loads, exports every entry point include/nvgs.h declares,
the Python binding's struct layouts match the C compiler's, and argument validation works
without a GPU (no compute call is made here)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nvgs.h")


@pytest.fixture(scope="module")
def N():
    from paper_2511_19202_b300 import build
    build.build()
    from paper_2511_19202_b300 import nvgs
    return nvgs


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nvgs_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(N):
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nvgs_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert set(N.EXPORTS) == set(declared)


def test_struct_layouts_match_the_c_compiler(N):
    structs = {"nvgs_asset_desc": N.AssetDesc, "nvgs_instance": N.Instance,
               "nvgs_camera": N.Camera, "nvgs_render_flags": N.RenderFlags,
               "nvgs_frame_stats": N.FrameStats, "nvgs_frame_view": N.FrameView,
               "nvgs_kernel_stat": N.KernelStat, "nvgs_asset_info": N.AssetInfo,
               "nvgs_train_batch": N.TrainBatch, "nvgs_adam_cfg": N.AdamCfg,
               "nvgs_asset_grads": N.AssetGrads, "nvgs_batch_opts": N.BatchOpts,
               "nvgs_tune_result": N.TuneResult, "nvgs_view_opts": N.ViewOpts,
               "nvgs_view_instances": N.ViewInstances}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-o", exe, c], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_default_flags_are_the_papers_constants(N):
    f = N.nvgs_default_flags()
    assert f.alpha_min == pytest.approx(1 / 255) and f.t_stop == pytest.approx(1e-4)
    assert f.alpha_max == pytest.approx(0.99) and f.dilation == pytest.approx(0.3)
    assert f.tile_size == 16 and f.use_mlp == 1 and f.logit_threshold == 0.0
    assert N.nvgs_abi_version() == 1


def test_create_fails_cleanly_on_a_bad_device(N):
    h = C.c_void_p()
    st = N.lib.nvgs_create(C.byref(h), 9999, None)
    assert st != N.NVGS_OK and not h.value
    assert N.lib.nvgs_create(None, 0, None) == N.NVGS_ERR_INVALID_ARG
    assert N.lib.nvgs_destroy(None) == N.NVGS_ERR_INVALID_ARG
    g = N.AssetGrads()
    assert N.lib.nvgs_render_backward(None, None, 0, C.byref(g)) == N.NVGS_ERR_INVALID_ARG
    assert N.lib.nvgs_update_asset(None, 0, None, None, None, None, None) == N.NVGS_ERR_INVALID_ARG
    assert N.lib.nvgs_render_batch(None, None, 0, None, None, None, None) == N.NVGS_ERR_INVALID_ARG
    assert N.lib.nvgs_render_views(None, None, None, 0, None, None, None, None) == N.NVGS_ERR_INVALID_ARG
