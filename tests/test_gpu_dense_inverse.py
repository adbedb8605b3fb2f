"""The capacitance inversion kernel (blocked Gauss-Jordan with partial pivoting, Sec. 4.4's dense
contact-space solve) against a plain dense inverse, across its storage modes and ragged sizes:
columns in shared memory, in global memory, and narrow panels for n > 2048; FP64 and FP32."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_16478_gb300 import Context
    return Context(0)


def _capacitance_like(n, seed):
    """I + K D with D symmetric positive definite and K block-diagonal 3x3 lower-triangular with a
    wide spread of magnitudes (sticking, sliding and nearly separated contacts)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) / np.sqrt(n)
    D = X @ X.T + 0.05 * np.eye(n)
    K = np.zeros((n, n))
    for c in range(0, n, 3):
        b = min(3, n - c)
        blk = np.tril(rng.standard_normal((b, b)))
        blk[np.diag_indices(b)] = np.abs(blk[np.diag_indices(b)]) * 10.0 ** rng.uniform(-6, 2)
        K[c:c + b, c:c + b] = blk
    return np.eye(n) + K @ D


def _needs_pivoting(n, seed):
    """A row permutation of a well-conditioned matrix with zeros on the diagonal."""
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    perm = np.roll(np.arange(n), 1)
    B = A[perm]
    B[np.arange(n), np.arange(n)] = 0.0
    return B


def _check(ctx, M, precision, tol):
    from paper_2603_16478_gb300.binding import dense_inverse
    Cm = torch.tensor(M, dtype=torch.float64, device="cuda")
    Ci = dense_inverse(ctx, Cm, precision).cpu().numpy()
    ref = np.linalg.inv(M)
    err = np.linalg.norm(Ci - ref) / np.linalg.norm(ref)
    assert err < tol, (M.shape[0], precision, err)
    return Ci


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 31, 64, 511, 512, 513, 1024, 1353, 1700, 2048, 2049, 3001])
def test_fp64_inverse(ctx, n):
    M = _capacitance_like(n, n)
    cond = np.linalg.cond(M)
    _check(ctx, M, "fp64", 2e-16 * n * max(cond, 1.0) + 1e-13)


@pytest.mark.parametrize("n", [1, 17, 100, 1353, 2048, 2600, 4096, 4097, 6990, 8192, 8193, 9500])
def test_fp32_inverse(ctx, n):
    rng = np.random.default_rng(n + 7)
    M = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    # |G/sqrt(n)| ~ 2 for a Gaussian G, so cond(M) <= ~5 (computed exactly only where it is cheap)
    cond = np.linalg.cond(M) if n <= 2048 else 6.0
    _check(ctx, M, "mixed", 5e-7 * cond * np.sqrt(n))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [5, 300, 1353])
def test_row_pivoting(ctx, n, precision):
    M = _needs_pivoting(n, n)
    _check(ctx, M, precision, 1e-12 if precision == "fp64" else 1e-4)


def test_repeat_calls_are_deterministic(ctx):
    from paper_2603_16478_gb300.binding import dense_inverse
    M = torch.tensor(_capacitance_like(1353, 3), device="cuda")
    a = dense_inverse(ctx, M, "fp64")
    b = dense_inverse(ctx, M, "fp64")
    assert torch.equal(a, b)
    c = dense_inverse(ctx, M, "mixed")
    d = dense_inverse(ctx, M, "mixed")
    assert torch.equal(c, d)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_singular_matrix_is_reported_and_the_next_call_works(ctx, precision):
    from paper_2603_16478_gb300.binding import NcpadjError, dense_inverse
    n = 700
    M = _capacitance_like(n, 11)
    M[:, 123] = 0.0  # an all-zero column: no pivot exists at that step
    with pytest.raises(NcpadjError, match="NONFINITE"):
        dense_inverse(ctx, torch.tensor(M, device="cuda"), precision)
    good = _capacitance_like(n, 12)
    _check(ctx, good, precision, 1e-10 if precision == "fp64" else 1e-3)


def test_invalid_sizes_are_rejected(ctx):
    from paper_2603_16478_gb300.binding import NcpadjError, dense_inverse
    with pytest.raises(NcpadjError, match="INVALID_ARG"):
        dense_inverse(ctx, torch.zeros(16385, 1, dtype=torch.float64, device="cuda").expand(16385, 16385))
    with pytest.raises(NcpadjError, match="UNSUPPORTED"):  # FP64 panels stop at 4096 rows
        dense_inverse(ctx, torch.eye(4097, dtype=torch.float64, device="cuda"), "fp64")


def test_alternating_sizes_and_precisions_share_one_workspace(ctx):
    """Inversions of different sizes and precisions one after another reuse the same scratch;
    each must start from clean synchronisation flags."""
    for n, prec in [(3001, "fp64"), (1, "mixed"), (2600, "mixed"), (7, "fp64"), (1353, "mixed"), (1353, "fp64"),
                    (40, "mixed"), (2049, "fp64")]:
        rng = np.random.default_rng(n)
        M = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
        _check(ctx, M, prec, (1e-12 if prec == "fp64" else 1e-5) * np.linalg.cond(M) * np.sqrt(n))


# ---- the blocked Gauss-Jordan on the tensor cores (NCPADJ_TF32X3) ---------------------------

@pytest.mark.parametrize("n", [1, 5, 63, 64, 65, 127, 128, 129, 200, 1353, 2088, 3001])
def test_tensor_core_blocked_inverse(ctx, n):
    """FP32 storage, 3xTF32 rank-64 updates: the result is within FP32 rounding of the inverse
    (well-conditioned matrices whose diagonal blocks stay invertible); ragged last blocks and tiles."""
    rng = np.random.default_rng(n + 11)
    M = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    cond = np.linalg.cond(M) if n <= 2048 else 6.0
    _check(ctx, M, "tf32x3", 2e-6 * cond * np.sqrt(n))


@pytest.mark.parametrize("n", [300, 1353, 2088])
def test_tensor_core_inverse_of_capacitance_like_matrices(ctx, n):
    """The capacitance structure I + K D (3 x 3 contact blocks of widely spread magnitude): as a
    preconditioner the result must leave ||I - M B|| small, like the pivoted Gauss-Jordan's."""
    from paper_2603_16478_gb300.binding import dense_inverse
    M = _capacitance_like(n, n + 1)
    Cm = torch.tensor(M, dtype=torch.float64, device="cuda")
    res = {}
    for prec in ("mixed", "tf32x3"):
        B = dense_inverse(ctx, Cm, prec).cpu().numpy()
        res[prec] = np.linalg.norm(np.eye(n) - M @ B) / np.sqrt(n)
    assert res["tf32x3"] < max(1e-3, 20 * res["mixed"]), res


def test_tensor_core_inverse_pivots_inside_diagonal_blocks(ctx):
    """Zeros on the diagonal inside every 64 x 64 block: the block's own row pivoting handles them."""
    n = 300
    rng = np.random.default_rng(5)
    M = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    perm = np.arange(n)
    for b0 in range(0, n, 64):  # rotate the rows within each diagonal block
        blk = perm[b0:min(n, b0 + 64)]
        perm[b0:min(n, b0 + 64)] = np.roll(blk, 1)
    M = M[perm]
    M[np.arange(n), np.arange(n)] = 0.0
    _check(ctx, M, "tf32x3", 1e-4)


def test_tensor_core_inverse_repeat_calls_are_deterministic(ctx):
    from paper_2603_16478_gb300.binding import dense_inverse
    M = torch.tensor(_capacitance_like(1353, 3), device="cuda")
    a = dense_inverse(ctx, M, "tf32x3")
    b = dense_inverse(ctx, M, "tf32x3")
    assert torch.equal(a, b)


def test_tensor_core_inverse_needs_invertible_diagonal_blocks(ctx):
    """Pivoting stays inside the 64 x 64 diagonal blocks: a matrix whose leading block is singular
    is reported (NONFINITE), not returned as garbage, and the next call works."""
    from paper_2603_16478_gb300 import NcpadjError
    from paper_2603_16478_gb300.binding import dense_inverse
    n = 100
    rng = np.random.default_rng(1)
    M = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    M[:64, :64] = 0.0  # the leading 64 x 64 block is zero
    M[:64, 64:] = rng.standard_normal((64, 36))
    with pytest.raises(NcpadjError, match="NONFINITE"):
        dense_inverse(ctx, torch.tensor(M, device="cuda"), "tf32x3")
    good = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    _check(ctx, good, "tf32x3", 1e-5)
