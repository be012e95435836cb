"""adp_lower_solve_noalloc: the lower-level solve for callers that cannot
allocate device memory where they need it (cudaMalloc/cudaFree synchronise the
device; some callers own all device memory through their own pool).

Its workspace is a fixed array inside the library, shared by every call, so the
checks run two calls in a row on the same inputs: each must match the regular
adp_lower_solve (which allocates its workspace when the problem is created).
This file is collected last so that a failure here leaves every other test
already run; it also passes when run alone in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp, synth
from gpu_common import need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("C,H,W,K,prec,eps", [(3, 70, 45, 7, adp.ADP_F32, 1e-2),
                                              (3, 256, 256, 15, adp.ADP_F32, 1e-2),
                                              (1, 64, 64, 7, adp.ADP_F64, 1e-4)])
def test_noalloc_matches_lower_solve_on_two_calls(C, H, W, K, prec, eps):
    need_gpu()
    inst = synth.make_instance("na", C, H, W, synth.gaussian_kernel(K, K / 5.0), synth.gaussian_kernel(K, K / 6.0),
                               0.01, 3)
    dt = torch.float32 if prec == adp.ADP_F32 else torch.float64
    params = adp.Params(C, H, W, K, prec=prec)
    y = torch.tensor(inst.y, dtype=dt, device="cuda")
    a = torch.tensor(inst.a, dtype=dt, device="cuda")
    b = torch.tensor(inst.b_true, dtype=dt, device="cuda")
    prob = adp.Problem(params, y, a)
    x_ref = y.clone()
    it_ref, gn_ref, cap_ref = prob.lower_solve(b, x_ref, eps, 300)
    torch.cuda.synchronize()

    lib = adp.load_library()
    cp = params.c()
    stream = torch.cuda.current_stream()
    tol = 1e-6 if prec == adp.ADP_F32 else 1e-12
    for call in range(2):
        x = y.clone()
        it, gn = ct.c_int(), ct.c_double()
        st = lib.adp_lower_solve_noalloc(ct.byref(cp), ct.c_void_p(y.data_ptr()), ct.c_void_p(b.data_ptr()),
                                         ct.c_void_p(x.data_ptr()), float(eps), 300, ct.c_void_p(stream.cuda_stream),
                                         ct.byref(it), ct.byref(gn))
        assert st in (adp.ADP_OK, adp.ADP_ENOCONV), lib.adp_last_error().decode()
        assert (st == adp.ADP_ENOCONV) == cap_ref
        assert it.value == it_ref, (call, it.value, it_ref)
        assert gn.value == pytest.approx(gn_ref, rel=tol)
        assert rel(x.double().cpu().numpy(), x_ref.double().cpu().numpy()) <= tol, call


def test_noalloc_rejects_images_beyond_its_limit():
    need_gpu()
    C, H, W, K = 3, 640, 640, 5        # 3 * 640 * 640 * 4 bytes > ADP_NOALLOC_MAX_IMAGE_BYTES
    params = adp.Params(C, H, W, K)
    y = torch.zeros((C, H, W), device="cuda")
    b = torch.zeros((C, K, K), device="cuda")
    with pytest.raises(adp.AdpError) as e:
        adp.adp_lower_solve_noalloc(params, y, b, y.clone(), 1e-2)
    assert e.value.status == adp.ADP_EINVAL
    assert "no-allocation limit" in str(e.value)
