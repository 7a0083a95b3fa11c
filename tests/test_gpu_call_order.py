"""Call order and argument errors of the C ABI on a live context.

Every PC_ESTATE and PC_EINVAL case that include/phononic.h documents for pc_bands,
pc_gap_and_grad, pc_gap_ks_and_grad, pc_apply_operator, pc_export and pc_import_block returns
its code before anything is enqueued, and the context still gives the oracle's bands (Results,
eq. matrixform) afterwards.  A gradient is never formed from the eigenvectors of an earlier
design: pc_set_design clears the band results, so pc_gap_and_grad refuses until pc_bands has
run on the new design.  SC 8^3 binary cube, M = 1, 10 k, 6 bands, both forms.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import mixed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = {"fp64": 1e-9, "mixed": 1e-6}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_06855_gb300 import binding, build_lib
    build_lib.build()
    binding.load()
    return binding


def _code(B, fn, *args):
    with pytest.raises(B.PhononicError) as e:
        fn(*args)
    return e.value.code


def _omega_err(w_gpu, w_ref):
    """Floored relative frequency error; the Gamma zero modes (lambda <= 1e-9 lambda_max on the
    reference side) are checked on lambda instead."""
    lam_ref = w_ref ** 2
    zero = lam_ref <= 1e-9 * lam_ref.max()
    assert np.all(w_gpu[zero] ** 2 <= 1e-9 * lam_ref.max())
    err = np.abs(w_gpu - w_ref) / np.maximum(w_ref, 0.05 * w_ref.max())
    return np.max(np.where(zero, 0.0, err))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_call_order_and_argument_errors(B, precision):
    w = wl.sc8_binary_cube()
    prec = B.PC_FP64 if precision == "fp64" else B.PC_MIXED
    ctx = B.pc_create(B.make_params(w.lattice, w.n, w.M, w.nbands, w.phase1, w.phase0, w.penal, prec, w.a))
    try:
        dev = torch.device("cuda")
        s = torch.cuda.current_stream(dev).cuda_stream
        nk, nb = len(w.Q), w.nbands
        N = (2 * w.M + 1) ** 3
        om = torch.empty((nk, nb), dtype=torch.float64, device=dev)
        gap = torch.empty(1, dtype=torch.float64, device=dev)
        grad = torch.empty(w.n, dtype=torch.float64, device=dev)
        x = torch.zeros((2, 3 * N), dtype=torch.complex128, device=dev)
        ax, ox = torch.empty_like(x), torch.empty_like(x)
        rho = torch.from_numpy(w.rho.ravel().copy()).to(dev)
        OM = B.PC_GAP_OMEGA

        def gap_rc(n_lower, mode=OM, wptr=0):
            return _code(B, B.pc_gap_and_grad, ctx, n_lower, mode, wptr, gap.data_ptr(), grad.data_ptr(), s)

        def ks_rc(n_lower, beta):
            return _code(B, B.pc_gap_ks_and_grad, ctx, n_lower, beta, gap.data_ptr(), grad.data_ptr(), s)

        def apply_rc(k, ncols):
            return _code(B, B.pc_apply_operator, ctx, k, ncols, x.data_ptr(), ax.data_ptr(), ox.data_ptr(), s)

        # neither k-points nor a design
        assert _code(B, B.pc_bands, ctx, om.data_ptr(), s) == B.PC_ESTATE
        assert _code(B, B.pc_export, ctx, B.PC_EXPORT_SFAC) == B.PC_ESTATE
        assert _code(B, B.pc_import_block, ctx, np.zeros(8)) == B.PC_ESTATE
        B.pc_set_kpoints(ctx, np.ascontiguousarray(w.Q))
        # k-points, no design
        assert _code(B, B.pc_bands, ctx, om.data_ptr(), s) == B.PC_ESTATE
        assert apply_rc(0, 2) == B.PC_ESTATE
        for which in (B.PC_EXPORT_SFAC, B.PC_EXPORT_TOEP, B.PC_EXPORT_WINV):
            assert _code(B, B.pc_export, ctx, which) == B.PC_ESTATE
        B.pc_set_design(ctx, rho.data_ptr(), s)
        # design, no bands
        assert gap_rc(3) == B.PC_ESTATE
        assert ks_rc(3, 10.0) == B.PC_ESTATE
        for which in (B.PC_EXPORT_LAMBDA, B.PC_EXPORT_EIGVEC, B.PC_EXPORT_WEIGHT, B.PC_EXPORT_BLOCK):
            assert _code(B, B.pc_export, ctx, which) == B.PC_ESTATE
        B.pc_bands(ctx, om.data_ptr(), s)
        first = om.cpu().numpy().copy()
        # argument errors with the bands in place
        for n_lower in (0, -1, nb):
            assert gap_rc(n_lower) == B.PC_EINVAL
            assert ks_rc(n_lower, 10.0) == B.PC_EINVAL
        assert gap_rc(3, mode=7) == B.PC_EINVAL
        assert gap_rc(3, mode=B.PC_GRAD_ALLBANDS, wptr=0) == B.PC_EINVAL
        for beta in (0.0, -1.0, 1e12, float("nan"), float("inf")):
            assert ks_rc(3, beta) == B.PC_EINVAL
        for k, ncols in ((-1, 2), (nk, 2), (0, 0), (0, 10 ** 6)):
            assert apply_rc(k, ncols) == B.PC_EINVAL
        assert _code(B, B.pc_export, ctx, 99) == B.PC_EINVAL
        assert _code(B, B.pc_import_block, ctx, np.zeros(8)) == B.PC_EINVAL
        # the refused calls left the context usable: a gap and gradient, then a new design
        B.pc_gap_and_grad(ctx, 3, OM, 0, gap.data_ptr(), grad.data_ptr(), s)
        torch.cuda.synchronize()
        assert np.isfinite(gap.item()) and bool(torch.isfinite(grad).all())
        other = torch.from_numpy(np.clip(w.rho.ravel() * 0.5 + 0.25, 0.0, 1.0)).to(dev)
        B.pc_set_design(ctx, other.data_ptr(), s)
        assert gap_rc(3) == B.PC_ESTATE  # no gradient from the previous design's eigenvectors
        assert ks_rc(3, 10.0) == B.PC_ESTATE
        B.pc_set_design(ctx, rho.data_ptr(), s)
        B.pc_bands(ctx, om.data_ptr(), s)
        again = om.cpu().numpy()
        assert B.pc_get_stats(ctx).status == B.PC_OK
        ref = mixed.omega(mixed.bands(mixed.from_workload(w), w.Q, nb))
        assert _omega_err(first, ref) <= TOL_W[precision]
        assert _omega_err(again, ref) <= TOL_W[precision]
    finally:
        B.pc_destroy(ctx)
