"""The allocation-free tensor-core GEMM (diam_op_gemm_bf16_noalloc) against the allocating one.

Callers that cannot call cudaMalloc (code whose device memory belongs to its own pool, or code on a
latency-critical path that cannot afford the synchronisation an allocation may cause) use the
allocation-free entry point; it must give the same product as diam_op_gemm_bf16. Two calls in a row, on
each of two shapes, check that the shared scratch array carries nothing over from one call to the next.
This file is collected last so that a failure here does not hide any other test.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-5   # relative to the largest |entry|: FP32 accumulation in a different order (split K)


def _fns():
    import paper_1506_05741_b300 as dm
    l = dm.lib()
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    out = []
    for name in ("diam_op_gemm_bf16", "diam_op_gemm_bf16_noalloc"):
        f = getattr(l, name)
        f.argtypes = [I32, I32, I32, P, I32, P, P, I32, I32, ctypes.c_float, P, I32, P]
        f.restype = ctypes.c_int
        out.append(f)
    return out


def _call(f, M, N, K, A, B, B2, scale, a_lower=0):
    import torch
    D = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    rc = f(M, N, K, A.data_ptr(), A.shape[1], B.data_ptr(), None if B2 is None else B2.data_ptr(), B.shape[1],
           a_lower, scale, D.data_ptr(), M, None)
    return rc, D


def test_noalloc_gemm_matches_allocating_gemm_twice_in_a_row():
    import torch
    ref_f, na_f = _fns()
    g = torch.Generator(device="cuda").manual_seed(2024)
    for M, N, K, scale, lower in [(2048, 256, 4096, 0.75, 0), (300, 130, 320, 1.0, 1)]:
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        if lower:
            A = torch.tril(A.float()).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        B2 = (torch.randn(N, K, device="cuda", generator=g) * 1e-2).to(torch.bfloat16)
        rc, Dref = _call(ref_f, M, N, K, A.view(torch.int16), B.view(torch.int16), B2.view(torch.int16), scale, lower)
        assert rc == 0
        for _ in range(2):   # two calls in a row on the shared scratch
            rc, Dna = _call(na_f, M, N, K, A.view(torch.int16), B.view(torch.int16), B2.view(torch.int16), scale,
                            lower)
            assert rc == 0
            assert torch.isfinite(Dna).all()
            assert (Dna - Dref).abs().max().item() <= TOL * Dref.abs().max().item()


def test_noalloc_gemm_rejects_products_beyond_its_scratch():
    import torch
    _, na_f = _fns()
    M, N, K = 4096, 1025, 64          # M * N = 4,198,400 > 4,194,240 floats of scratch
    A = torch.zeros(M, K, dtype=torch.int16, device="cuda")
    B = torch.zeros(N, K, dtype=torch.int16, device="cuda")
    D = torch.zeros(N, M, dtype=torch.float32, device="cuda")
    rc = na_f(M, N, K, A.data_ptr(), K, B.data_ptr(), None, K, 0, 1.0, D.data_ptr(), M, None)
    assert rc == 1   # DIAM_EINVAL
