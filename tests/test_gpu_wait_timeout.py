"""Device self-checks.  Failure path of the bounded device-side waits (the tensor-core MLP kernels' mbarrier waits): a
wait on an mbarrier that nothing arrives on gives up after about a second, the kernel records it
and returns, and the context stays usable -- a render afterwards matches one before."""
import pytest

import scenes
from gpu_common import renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_the_context_survives():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.tiny_scene(2000, 2, sh_degree=1)
    cam = scenes.look_at_camera((0.0, 0.5, 3.0), (0, 0, 0), 96, 64, 50.0)
    r = renderer_for(sc)
    try:
        before, _ = r.render(cam, r.flags(use_mlp=0))
        before = before.clone()
        status, seconds = N.nvgs_selftest_wait_timeout(0)
        assert status == N.NVGS_OK
        assert 0.1 < seconds < 5.0, seconds
        after, _ = r.render(cam, r.flags(use_mlp=0))
        assert torch.equal(before, after)
    finally:
        r.close()


def test_fp32_fma_throughput_is_measured():
    """The ALU roofline's denominator: FP32 FMA throughput measured on the device (a B300 runs
    148 SMs x 128 FP32 lanes x 2 flops per clock, ~77 TFLOP/s at 2032 MHz)."""
    from paper_2511_19202_b300 import nvgs as N
    t = N.nvgs_measure_fp32_fma(0)
    print(f"FP32 FMA: {t:.1f} TFLOP/s")
    assert 5.0 < t < 200.0


def test_failed_allocation_is_reported_and_the_context_recovers():
    """Host-side fault injection: buffer growths fail as out-of-memory; the render that needs
    them returns NVGS_ERR_OOM with a message, and once the fault is lifted the same context
    renders the frame exactly as a fresh context does."""
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.tiny_scene(3000, 3, sh_degree=1)
    small = scenes.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 48, 32, 50.0)
    big = scenes.look_at_camera((0.0, 0.3, 2.0), (0, 0, 0), 320, 240, 60.0)
    r = renderer_for(sc)
    try:
        r.render(small, r.flags(use_mlp=0))
        N.nvgs_debug_fail_allocs(1000)
        try:
            with pytest.raises(N.NvgsError) as e:
                r.render(big, r.flags(use_mlp=0))
            assert e.value.status == N.NVGS_ERR_OOM
        finally:
            N.nvgs_debug_fail_allocs(0)
        img, _ = r.render(big, r.flags(use_mlp=0))
        img = img.clone()
    finally:
        r.close()
    r2 = renderer_for(sc)
    try:
        ref, _ = r2.render(big, r2.flags(use_mlp=0))
        assert torch.equal(img, ref)
    finally:
        r2.close()
