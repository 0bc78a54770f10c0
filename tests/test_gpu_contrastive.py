"""GPU parity of the contrastive (InfoNCE) join against the FP64 oracle.

The GPU computes on BF16 roundings of the float32 inputs with FP32
accumulation; the oracle evaluates the same BF16 values in FP64.  Tolerances
(derived from the arithmetic): forward values carry FP32 accumulation and an
approximate exp2 (relative ~1e-6 of |S| <= 1/T), so lse and loss agree to a
few 1e-5 absolute.  The backward feeds dL/dS tiles rounded to BF16 (relative
error <= 2^-8) to the tensor cores and accumulates N products in FP32, so each
gradient entry is held to the bound derived from that arithmetic,
  |dA_ik - ref| <= (g / (N T)) sum_j [(2^-8 + (N + 64) 2^-22 + 1e-5) |G'_ij|
                                       + P_ij (|dl_i| + 1e-6)] |b_jk|,
(G' = P - I, plus the column term when symmetric), where dl_i is the
measured error of the forward's logsumexp the backward consumes (it scales
every P_ij of the row by exp(dl_i)), and the gradient as a whole to a cosine
of 0.999 with the reference.
"""
import numpy as np
import pytest

import oracle
from paper_2112_07552_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf16_inputs(A, B):
    a = torch.from_numpy(A).to(torch.bfloat16)
    b = torch.from_numpy(B).to(torch.bfloat16)
    bits = lambda t: t.view(torch.int16).numpy().view(np.uint16)
    return bits(a), bits(b)


def run(sjmod, A, B, T, sym=False, g=1.0, fused=False):
    """fused: the backward recomputes dL/dS per output chunk instead of
    writing it and its transpose to memory (the default when they fit)."""
    d = A.shape[1]
    flags = sjmod.SJ_FLAG_SYM_INFONCE if sym else 0
    if fused:
        flags |= sjmod.SJ_FLAG_FUSED_BACKWARD
    with sjmod.SimilarityJoin(d, prec="bf16", device=0, flags=flags) as J:
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda()
        loss, lse = J.contrastive_forward(dA, dB, T)
        gA, gB = J.contrastive_backward(dA, dB, T, lse, torch.tensor([g], device="cuda"))
        torch.cuda.synchronize()
    return float(loss.item()), lse.cpu().numpy(), gA.cpu().numpy(), gB.cpu().numpy()


def grad_bounds(ab, bb, T, sym, g, dl_row=None, dl_col=None):
    """Per-entry error bounds of dA and dB (see the module docstring).

    dl_row / dl_col: measured |lse_gpu - lse_ref| per row / column (or None).
    """
    A = oracle.bf16_bits_to_f64(ab) if ab.dtype == np.uint16 else ab.astype(np.float64)
    B = oracle.bf16_bits_to_f64(bb) if bb.dtype == np.uint16 else bb.astype(np.float64)
    N = A.shape[0]
    S = A @ B.T / T
    I = np.eye(N)
    lr = S.max(axis=1, keepdims=True)
    P = np.exp(S - lr)
    P /= P.sum(axis=1, keepdims=True)
    G = P - I
    dlr = (np.zeros(N) if dl_row is None else np.asarray(dl_row)) + 1e-6
    E = P * dlr[:, None]          # propagated lse error of the row softmax
    if sym:
        lc = S.max(axis=0, keepdims=True)
        Q = np.exp(S - lc)
        Q /= Q.sum(axis=0, keepdims=True)
        G = 0.5 * (G + Q - I)
        dlc = (np.zeros(N) if dl_col is None else np.asarray(dl_col)) + 1e-6
        E = 0.5 * (E + Q * dlc[None, :])
    c = (2.0 ** -8 + (N + 64) * 2.0 ** -22 + 1e-5)
    W = c * np.abs(G) + E
    s = abs(g) / (N * T)
    return s * (W @ np.abs(B)), s * (W.T @ np.abs(A))


def check_grad(got, want, bound=None):
    got = got.astype(np.float64)
    cos = got.ravel() @ want.ravel() / (np.linalg.norm(got) * np.linalg.norm(want))
    assert cos >= 0.999, cos
    if bound is not None:
        err = np.abs(got - want)
        worst = np.max(err / (bound + 1e-30))
        assert worst <= 1.0, worst


@pytest.fixture(scope="module")
def sjmod():
    from paper_2112_07552_gb300 import _build, sj
    _build.build()
    return sj


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("N,d,T", [(64, 32, 0.05), (100, 100, 0.1), (300, 64, 0.05),
                                   (257, 200, 0.2), (640, 448, 0.05)])
def test_contrastive_matches_oracle(sjmod, N, d, T, sym, fused):
    A, B = datagen.paired(N, d, max(2, N // 8), seed=N + d)
    ab, bb = bf16_inputs(A, B)
    loss_w, lse_w, lsec_w, dA_w, dB_w = oracle.infonce(ab, bb, T, sym=sym, g=0.7)
    loss, lse, gA, gB = run(sjmod, A, B, T, sym=sym, g=0.7, fused=fused)
    assert abs(loss - loss_w) <= 5e-5 * max(1.0, abs(loss_w))
    assert np.max(np.abs(lse[:N] - lse_w)) <= 5e-5 * max(1.0, np.max(np.abs(lse_w)))
    if sym:
        assert np.max(np.abs(lse[N:] - lsec_w)) <= 5e-5 * max(1.0, np.max(np.abs(lsec_w)))
    bA, bB = grad_bounds(ab, bb, T, sym, 0.7, np.abs(lse[:N] - lse_w),
                         np.abs(lse[N:] - lsec_w) if sym else None)
    check_grad(gA, dA_w, bA)
    check_grad(gB, dB_w, bB)


def test_identity_closed_form(sjmod):
    # A = B = I (d = N): L = log(e^{1/T} + N - 1) - 1/T; dL/dS has a closed form
    N, T = 128, 0.5
    I = np.eye(N, dtype=np.float32)
    loss, lse, gA, gB = run(sjmod, I, I, T)
    Z = np.exp(1.0 / T) + N - 1
    assert abs(loss - (np.log(Z) - 1.0 / T)) <= 1e-5
    G = np.full((N, N), 1.0 / Z)
    np.fill_diagonal(G, -(N - 1) / Z)
    G /= N
    bA, bB = grad_bounds(I, I, T, False, 1.0)
    check_grad(gA, G / T, bA)
    check_grad(gB, G.T / T, bB)


def test_finite_differences_64x64_d32(sjmod):
    # FP64 central differences of the oracle loss at the BF16-rounded inputs
    N, d, T = 64, 32, 0.05
    A, B = datagen.paired(N, d, 8, seed=41)
    ab, bb = bf16_inputs(A, B)
    A64, B64 = oracle.bf16_bits_to_f64(ab), oracle.bf16_bits_to_f64(bb)
    _, _, gA, gB = run(sjmod, A, B, T)
    bounds = grad_bounds(ab, bb, T, False, 1.0)
    rng = np.random.default_rng(0)
    h = 1e-6
    for X, g in ((A64, gA), (B64, gB)):
        fd = np.zeros_like(X)
        idx = [(int(rng.integers(N)), int(rng.integers(d))) for _ in range(60)]
        for i, k in idx:
            old = X[i, k]
            X[i, k] = old + h
            lp = oracle.infonce(A64, B64, T, grads=False)[0]
            X[i, k] = old - h
            lm = oracle.infonce(A64, B64, T, grads=False)[0]
            X[i, k] = old
            fd[i, k] = (lp - lm) / (2 * h)
        got = np.array([g[i, k] for i, k in idx])
        want = np.array([fd[i, k] for i, k in idx])
        bnd = np.array([bounds[X is B64][i, k] for i, k in idx]) + 1e-8  # + FD truncation
        cos = got @ want / (np.linalg.norm(got) * np.linalg.norm(want))
        assert cos >= 0.999 and np.all(np.abs(got - want) <= bnd)


def test_autograd_function(sjmod):
    N, d, T = 200, 64, 0.1
    A, B = datagen.paired(N, d, 20, seed=43)
    ab, bb = bf16_inputs(A, B)
    loss_w, _, _, dA_w, dB_w = oracle.infonce(ab, bb, T, g=1.0)
    J = sjmod.SimilarityJoin(d, prec="bf16", device=0)
    tA = torch.from_numpy(A).cuda().requires_grad_()
    tB = torch.from_numpy(B).cuda().requires_grad_()
    loss = sjmod.contrastive_loss(tA, tB, T, J)
    loss.backward()
    assert abs(loss.item() - loss_w) <= 5e-5 * max(1.0, abs(loss_w))
    bA, bB = grad_bounds(ab, bb, T, False, 1.0)
    check_grad(tA.grad.cpu().numpy(), dA_w, bA)
    check_grad(tB.grad.cpu().numpy(), dB_w, bB)
    J.close()


def test_contrastive_debug_timeout(sjmod):
    A, B = datagen.paired(128, 64, 8, seed=44)
    J = sjmod.SimilarityJoin(64, prec="bf16", device=0, flags=sjmod.SJ_FLAG_DEBUG_TIMEOUT)
    with pytest.raises(sjmod.SJError) as e:
        J.contrastive_forward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 0.05)
    assert e.value.code == sjmod.SJ_ERR_TIMEOUT
    J.close()
    # the context stays usable
    loss, _, _, _ = run(sjmod, A, B, 0.05)
    assert np.isfinite(loss)


@pytest.fixture(scope="module")
def case_8192():
    N, d, T = 8192, 768, 0.05
    A, B = datagen.paired(N, d, 1000, seed=45)
    ab, bb = bf16_inputs(A, B)
    return A, B, ab, bb, T, oracle.infonce(ab, bb, T, g=1.0)


@pytest.mark.parametrize("fused", [False, True])
def test_contrastive_8192_full(sjmod, case_8192, fused):
    # every output against the oracle at N = 8,192, d = 768 (64 x 64 score
    # tiles, two output chunks of 384)
    A, B, ab, bb, T, want = case_8192
    loss_w, lse_w, _, dA_w, dB_w = want
    loss, lse, gA, gB = run(sjmod, A, B, T, fused=fused)
    assert abs(loss - loss_w) <= 5e-5 * max(1.0, abs(loss_w))
    assert np.max(np.abs(lse - lse_w)) <= 5e-5 * max(1.0, np.max(np.abs(lse_w)))
    bA, bB = grad_bounds(ab, bb, T, False, 1.0, np.abs(lse - lse_w))
    check_grad(gA, dA_w, bA)
    check_grad(gB, dB_w, bB)


def test_contrastive_65536_sampled_rows(sjmod):
    # the full-size join: row logsumexp and dA on sampled rows (each needs one
    # row of S only); dB needs every row's lse and is covered at N = 8,192
    N, d, T = 65536, 768, 0.05
    A, B = datagen.paired(N, d, 100_000, seed=0)
    ab, bb = bf16_inputs(A, B)
    loss, lse, gA, _ = run(sjmod, A, B, T)
    rows = np.sort(np.random.default_rng(7).choice(N, size=24, replace=False))
    lse_w, dA_w = oracle.infonce_rows(ab, bb, T, rows, g=1.0)
    assert np.max(np.abs(lse[rows] - lse_w)) <= 5e-5 * max(1.0, np.max(np.abs(lse_w)))
    # per-row bound as in grad_bounds, restricted to the sampled rows
    A64, B64 = oracle.bf16_bits_to_f64(ab[rows]), oracle.bf16_bits_to_f64(bb)
    S = A64 @ B64.T / T
    P = np.exp(S - lse_w[:, None])
    G = P.copy()
    G[np.arange(len(rows)), rows] -= 1.0
    c = 2.0 ** -8 + (N + 64) * 2.0 ** -22 + 1e-5
    W = c * np.abs(G) + P * (np.abs(lse[rows] - lse_w) + 1e-6)[:, None]
    check_grad(gA[rows], dA_w, (W @ np.abs(B64)) / (N * T))
    assert np.isfinite(loss)
