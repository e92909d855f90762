"""csff_norm2_noalloc: the allocation-free norm for callers that cannot
allocate device memory (their memory belongs to another allocator, or their
loop must not pay cudaMalloc's implicit synchronisation).  It is checked
through the C ABI against the plan-based csff_norm2 on the same vectors, on
two calls in a row (the fixed scratch array is shared between calls).

This file is collected last on purpose; it must pass on its own in a fresh
process and after the other tests."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-13   # both sides accumulate in FP64; only the summation order differs


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def _call(csff, v, out, exp_scale=0):
    arith = csff.ARITH_FP64 if v.dtype == torch.complex128 else csff.ARITH_FP32
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return csff._lib.csff_norm2_noalloc(arith, C.c_void_p(v.data_ptr()), C.c_longlong(v.numel()),
                                        int(exp_scale), C.c_void_p(out.data_ptr()), stream)


def test_noalloc_norm_matches_plan_norm_on_two_calls(csff):
    case = W.small_2d(n=129)
    plan = csff.Plan(case["problem"], case["opts"])
    N = plan.N
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    # call 1: FP64 vector; call 2: FP32 vector of another size, same shared scratch
    v1 = torch.from_numpy(W.rand_complex(N, 51, scale=7.0)).to("cuda")
    v2 = torch.from_numpy(W.rand_complex(N, 52, scale=0.3)).to("cuda").to(torch.complex64)
    assert _call(csff, v1, out[0:1]) == csff.OK
    assert _call(csff, v2, out[1:2]) == csff.OK
    torch.cuda.synchronize()
    ref1 = plan.norm2(0, v1)
    ref2 = plan.norm2(0, v2)
    got = out.cpu().numpy()
    assert abs(got[0] - ref1) <= TOL * ref1
    assert abs(got[1] - ref2) <= TOL * ref2
    # the same pair again: the scratch keeps the previous call's partials
    out2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(csff, v2, out2[1:2]) == csff.OK
    assert _call(csff, v1, out2[0:1]) == csff.OK
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), got)
    plan.close()


def test_noalloc_norm_prescale_and_limits(csff):
    big = torch.from_numpy(W.rand_complex(5000, 53, scale=1e200)).to("cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(csff, big, out, exp_scale=670) == csff.OK
    torch.cuda.synchronize()
    ref = np.linalg.norm(big.cpu().numpy() / 1e200) * 1e200
    assert abs(out.item() - ref) <= TOL * ref
    # beyond the fixed scratch: rejected before any launch, with a message
    st = csff._lib.csff_norm2_noalloc(csff.ARITH_FP64, C.c_void_p(big.data_ptr()), C.c_longlong((1 << 25) + 1),
                                      0, C.c_void_p(out.data_ptr()), None)
    assert st == csff.ERR_INVALID_ARG
    assert b"scratch limit" in csff._lib.csff_last_error()


def test_noalloc_norm_at_the_size_limit_through_the_wrapper(csff):
    """The largest allowed n (2^25 complex64 values: every one of the 4096
    partial slots in use), called through the Python wrapper, against a torch
    FP64 reference; further calls leave the device's free memory unchanged."""
    n = csff.NOALLOC_MAX_N
    g = torch.Generator(device="cuda").manual_seed(61)
    v = torch.randn(n, dtype=torch.complex64, device="cuda", generator=g)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    csff.norm2_noalloc(v, out)       # warm-up: the scratch address is looked up here
    torch.cuda.synchronize()
    ref = torch.sqrt(torch.sum(torch.view_as_real(v).double() ** 2)).item()
    assert abs(out.item() - ref) <= 1e-12 * ref
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        csff.norm2_noalloc(v, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert abs(out.item() - ref) <= 1e-12 * ref


def test_noalloc_wrapper_rejects_wrong_tensors(csff):
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        csff.norm2_noalloc(torch.zeros(16, dtype=torch.float32, device="cuda"), out)
    v = torch.zeros(32, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        csff.norm2_noalloc(v[::2], out)                   # strided view
    with pytest.raises(ValueError):
        csff.norm2_noalloc(v, torch.zeros(1, dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        csff.norm2_noalloc(v, torch.zeros(1, dtype=torch.float64))   # host tensor
