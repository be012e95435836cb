"""The BF16-operand tensor-core operator (adp_apply_B_bf16 / adp_apply_Bt_bf16)
against the FP64 oracle applied to the same BF16-rounded operands.

Every product of two BF16 values is exact in FP32, so the only error left is
the FP32 summation of the K^2 products of an output (4K steps of 16 products
each in tensor memory): tolerance relative L2 <= max(1e-6, 4 K u), u = 2^-24.
Shapes span several 128 x 32 output tiles with ragged tails in both
directions, widths that are not a multiple of four (the scalar store path), a
kernel wider than the image (the periodic wrap taken more than once) and the
degenerate K = 1.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_09758_gb300 import adp, synth
from gpu_common import Pair, need_gpu, rel

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


SHAPES = [(1, 40, 36, 5), (3, 130, 70, 15), (2, 257, 96, 31), (1, 8, 10, 33), (2, 33, 64, 1), (1, 129, 33, 3),
          (3, 256, 256, 15)]


def instance(C, H, W, K, seed):
    s = max(K / 5.0, 0.6)
    return synth.make_instance("bf16", C, H, W, synth.gaussian_kernel(K, 1.2 * s), synth.gaussian_kernel(K, s),
                               0.01, seed)


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_operators_match_oracle_on_rounded_operands(shape):
    C, H, W, K = shape
    pr = Pair(instance(C, H, W, K, 21 + K), prec=adp.ADP_F32)
    rng = np.random.default_rng(K)
    x = pr.rounded(rng.standard_normal((C, H, W)))
    b = pr.rounded(rng.standard_normal((C, K, K)) / K)
    xq, bq = oracle.bf16_round(x), oracle.bf16_round(b)
    tol = max(1e-6, 4 * K * U32)
    out = pr.n(pr.prob.apply_B_bf16(pr.t(b), pr.t(x)))
    assert rel(out, pr.P.conv(bq, xq)) <= tol
    outT = pr.n(pr.prob.apply_Bt_bf16(pr.t(b), pr.t(x)))
    assert rel(outT, pr.P.conv_adj(bq, xq)) <= tol
    assert pr.prob.bf16_grid_size() >= 1 and pr.prob.last_kernel_ms() > 0
    pr.prob.close()


def test_bf16_operator_is_the_bf16_one():
    """Against the FP32 operator the difference is the BF16 rounding of the
    operands (relative 2^-9 per value), well above FP32 rounding."""
    pr = Pair(instance(3, 96, 96, 15, 5), prec=adp.ADP_F32)
    rng = np.random.default_rng(1)
    x = pr.t(rng.standard_normal((3, 96, 96)))
    b = pr.t(rng.standard_normal((3, 15, 15)) / 15)
    d = rel(pr.n(pr.prob.apply_B_bf16(b, x)), pr.n(pr.prob.apply_B(b, x)))
    assert 1e-5 < d < 2.0 ** -7
    pr.prob.close()


def test_bf16_full_size_sampled():
    """512 x 512 RGB with K = 31 in the launch the library picks, sampled."""
    pr = Pair(synth.rgb512_k31(0), prec=adp.ADP_F32)
    C, H, W = pr.inst.shape
    K = pr.inst.K
    x = pr.rounded(pr.inst.x_true)
    b = pr.rounded(pr.inst.b_true)
    xq, bq = oracle.bf16_round(x), oracle.bf16_round(b)
    rng = np.random.default_rng(7)
    idx = [(c, i, j) for c in range(C) for i in (0, H - 1) for j in (0, W - 1)]
    idx += [(int(rng.integers(C)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(300)]
    out = pr.n(pr.prob.apply_B_bf16(pr.t(b), pr.t(x)))
    got = np.array([out[c, i, j] for c, i, j in idx])
    assert rel(got, pr.P.conv_at(bq, xq, idx)) <= max(1e-6, 4 * K * U32)
    outT = pr.n(pr.prob.apply_Bt_bf16(pr.t(b), pr.t(x)))
    got = np.array([outT[c, i, j] for c, i, j in idx])
    assert rel(got, pr.P.conv_adj_at(bq, xq, idx)) <= max(1e-6, 4 * K * U32)
    pr.prob.close()
    torch.cuda.empty_cache()


def test_bf16_rejects_unsupported_problems():
    p64 = Pair(instance(1, 16, 16, 5, 1), prec=adp.ADP_F64)
    z = p64.t(np.zeros((1, 16, 16)))
    with pytest.raises(adp.AdpError) as e:
        p64.prob.apply_B_bf16(p64.t(np.zeros((1, 5, 5))), z)
    assert e.value.status == adp.ADP_EINVAL
    p64.prob.close()
    big = Pair(instance(1, 64, 64, 35, 1), prec=adp.ADP_F32)
    with pytest.raises(adp.AdpError) as e:
        big.prob.apply_B_bf16(big.t(np.zeros((1, 35, 35))), big.t(np.zeros((1, 64, 64))))
    assert e.value.status == adp.ADP_EINVAL
    big.prob.close()


def test_bf16_problems_with_different_kernel_sizes_coexist():
    """A plan made later for a smaller K must not shrink what an earlier,
    larger plan launches with (the shared-memory attribute is per kernel)."""
    big = Pair(instance(1, 96, 64, 31, 3), prec=adp.ADP_F32)
    small = Pair(instance(1, 40, 32, 5, 4), prec=adp.ADP_F32)
    rng = np.random.default_rng(11)
    for pr, (C, H, W, K) in ((big, (1, 96, 64, 31)), (small, (1, 40, 32, 5)), (big, (1, 96, 64, 31))):
        x = pr.rounded(rng.standard_normal((C, H, W)))
        b = pr.rounded(rng.standard_normal((C, K, K)) / K)
        out = pr.n(pr.prob.apply_B_bf16(pr.t(b), pr.t(x)))
        assert rel(out, pr.P.conv(oracle.bf16_round(b), oracle.bf16_round(x))) <= max(1e-6, 4 * K * U32)
    big.prob.close()
    small.prob.close()
