"""Tensor-core kernels against CUDA-core references: those of the FP32 block iteration against the
FP32 CUDA-core kernels, and the sliced FP64-accurate products of the final Rayleigh-Ritz step
against the FP64 GEMM.

The batched Gram product A^H B and the basis update [S] C run on tcgen05 with both operands
split into three bf16 slices (six slice products, FP32 accumulation in tensor memory).  On
seeded data with column norms spread over 2^-3..2^3 they must agree with the CUDA-core FP32
kernels to 2e-5 of the largest result entry: both keep about 24 significant bits per operand
and accumulate in FP32, so the difference is a few FP32 roundings of sums of up to 4374 terms.
Sizes cover several 32-row stages and 128-row tiles with ragged tails, fewer rows than one
stage, block widths that are not multiples of 16, and one to three blocks per side.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


@pytest.mark.parametrize("nk,m,nblk,n3", [(3, 24, 3, 2187), (5, 10, 2, 75), (2, 16, 1, 33), (7, 24, 1, 1029),
                                          (150, 24, 3, 375)])
def test_gram_tensor_cores(B, nk, m, nblk, n3):
    err = B.pc_check_tensor_kernels(0, nk, m, nblk, n3)
    assert 0 <= err < TOL, err


@pytest.mark.parametrize("nk,m,nblk,n3", [(3, 24, 3, 2187), (5, 10, 2, 75), (2, 16, 1, 33), (4, 20, 3, 1029),
                                          (150, 24, 3, 375), (6, 8, 3, 130)])
def test_update_tensor_cores(B, nk, m, nblk, n3):
    err = B.pc_check_tensor_kernels(1, nk, m, nblk, n3)
    assert 0 <= err < TOL, err


def test_bounded_wait_expires(B):
    """Failure detection without a fault: a kernel waits on a barrier that nothing completes,
    with a short poll limit.  It must give up, record PC_ETIMEOUT in its status word and
    return, and the device must accept further work; the tensor-core kernels then still agree
    with the CUDA-core ones."""
    assert B.pc_check_tensor_kernels(2, 1, 1, 1, 1) == 0.0
    assert 0 <= B.pc_check_tensor_kernels(0, 2, 8, 1, 64) < TOL


@pytest.mark.parametrize("N,ncols", [(729, 300), (343, 70), (125, 33), (27, 5)])
def test_sliced_fp64_products(B, N, ncols):
    """The final Rayleigh-Ritz step's FP64-accurate products (exact 6-bit slices of both operands,
    36 slice products on the tensor cores, FP64 recombination) against the FP64 GEMM on seeded
    complex data whose operator rows span eight binades: 1e-10 of the largest result entry
    (measured about 2e-12 of the row and column scales; FP64 itself about 4e-15).  Sizes cover
    several 128-row and 64-column tiles with ragged tails and fewer rows than one tile."""
    err = B.pc_check_tensor_kernels(3, 1, ncols, 1, N)
    assert 0 <= err < 1e-10, err
