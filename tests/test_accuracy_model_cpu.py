"""CPU checks of the two accuracy facts the mixed precisions are built around (the
double-float energy rows, and the K-chunked tensor-core contractions):

1. With a small energy sigma, the few energy rows of the weighted design matrix steer
   the fitted forces: a relative perturbation of the energy rows moves the predicted
   forces far more than the same perturbation of the force rows (oracle matrices, exact
   least squares).
2. A dot product accumulated in FP32 with truncation toward zero after every step (how
   the tensor cores' accumulator behaves) drifts one-signed, toward zero, by an amount
   that grows with the number of steps; cutting the contraction into chunks of at most
   32 steps whose sums are added in round-to-nearest shrinks the drift (numpy emulation).
3. The force rows' products J_p . x_s from BF16 three-slice operands need all six
   products of slice order two or less: leaving out any of the order-two products
   leaves an error of order 2^-16 of the operands' scale, three orders of magnitude more
   than with all six, while FP16's scaled two-slice operands reach about 2^-22 with three
   products (exact accumulation here; the accumulator's truncation is fact 2).
"""
import numpy as np

import gapgen
import oracle


def _fit_forces(p, A, b, nE):
    c = np.linalg.lstsq(A, b, rcond=None)[0]
    return oracle.predict(p, c)[1]


def test_energy_rows_steer_the_forces_at_small_energy_sigma():
    r = gapgen.Recipe(n_cfg=40, atoms=(8, 24), d=24, n_sparse=(48,), zeta=2, neighbours=(4, 10),
                      sigma_e_atom=1e-4, seed=91)
    p = gapgen.make_problem(r)
    y = oracle.targets(p)
    A, _ = oracle.stacked_matrix(p)
    b = np.concatenate([y / oracle.sigma(p), np.zeros(p.n_sparse)])
    nE, N = p.n_cfg, p.n_rows
    F0 = _fit_forces(p, A, b, nE)
    rng = np.random.default_rng(3)
    eps = 1e-7
    Ae = A.copy()
    Ae[:nE] *= 1 + eps * rng.standard_normal(Ae[:nE].shape)
    Af = A.copy()
    Af[nE:N] *= 1 + eps * rng.standard_normal(Af[nE:N].shape)
    err_e = np.linalg.norm(_fit_forces(p, Ae, b, nE) - F0) / np.linalg.norm(F0)
    err_f = np.linalg.norm(_fit_forces(p, Af, b, nE) - F0) / np.linalg.norm(F0)
    assert err_e > 50 * err_f, (err_e, err_f)  # measured: 2.1e-6 against 7.8e-9


def _to_f32_toward_zero(x):
    f = x.astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(x)
    f[over] = np.nextafter(f[over], np.float32(0))
    return f


def _truncating_dot(a, b, steps, chunk=None):
    """sum_k a_k b_k over `steps` groups of 16 products: each group's sum exact, added to
    an FP32 accumulator truncated toward zero; with `chunk`, a new accumulator every
    `chunk` groups and the chunk sums added in FP32 round-to-nearest."""
    g = (a * b).reshape(a.shape[0], steps, -1).sum(axis=2)  # exact enough in FP64
    total = np.zeros(a.shape[0], np.float32)
    chunk = chunk or steps
    for c0 in range(0, steps, chunk):
        acc = np.zeros(a.shape[0], np.float32)
        for k in range(c0, min(steps, c0 + chunk)):
            acc = _to_f32_toward_zero(acc.astype(np.float64) + g[:, k])
        total = (total.astype(np.float64) + acc.astype(np.float64)).astype(np.float32)
    return total.astype(np.float64)


def test_truncating_accumulation_drifts_and_chunks_shrink_it():
    rng = np.random.default_rng(11)
    n, d = 4000, 2048
    a = rng.standard_normal((n, d)) * 0.1
    b = rng.random(d)
    b /= np.linalg.norm(b)
    exact = (a * b).sum(axis=1)

    def scale_error(steps, chunk=None):
        k = 16 * steps
        ex = (a[:, :k] * b[:k]).sum(axis=1)
        got = _truncating_dot(a[:, :k], np.broadcast_to(b[:k], a[:, :k].shape), steps, chunk)
        return float(np.sum(ex * (got - ex)) / np.sum(ex * ex))

    # measured here: -7.3e-7 at 32 steps, -2.8e-6 at 128, -7.0e-7 at 128 in chunks of 32
    # (the GB300's force rows: -2.2e-6 at 128 steps, -6.5e-7 in chunks of 32)
    e32, e128 = scale_error(32), scale_error(128)
    assert e32 < 0 and e128 < 0           # toward zero, one-signed
    assert e128 < 3 * e32                 # grows with the steps
    e128c = scale_error(128, chunk=32)
    assert e128c < 0 and abs(e128c) < 0.35 * abs(e128), (e128, e128c)
    assert exact.shape == (n,)


def _bf16(x):
    """Round to the nearest BF16 (ties to even), returned as FP64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_slices(x):
    s0 = _bf16(x)
    s1 = _bf16(x - s0)
    return s0, s1, _bf16(x - s0 - s1)


def _fp16_two_slice(x):
    """One power-of-two scale per row putting its largest magnitude in [2^14, 2^15), then
    x 2^e = f + g with f and g rounded to FP16."""
    e = 14 - np.floor(np.log2(np.abs(x).max(axis=1, keepdims=True)))
    xs = x * 2.0 ** e
    f = xs.astype(np.float16).astype(np.float64)
    return f, (xs - f).astype(np.float16).astype(np.float64), e


def test_force_products_need_six_bf16_slice_products():
    rng = np.random.default_rng(5)
    d = 512
    J = rng.normal(0.0, 0.1, (600, d))            # Jacobian rows as the workloads draw them
    Xs = np.abs(rng.normal(0.0, 1.0, (64, d)))     # normalised non-negative sparse points
    Xs /= np.linalg.norm(Xs, axis=1, keepdims=True)
    exact = J @ Xs.T
    a, b = _bf16_slices(J), _bf16_slices(Xs)

    def err(terms):
        approx = sum(a[i] @ b[j].T for i, j in terms)
        return np.linalg.norm(approx - exact) / np.linalg.norm(exact)
    first = [(0, 0), (0, 1), (1, 0)]
    six = err(first + [(0, 2), (1, 1), (2, 0)])
    assert six < 3e-8
    for extra in ([], [(1, 1)], [(0, 2), (2, 0)], [(0, 2), (1, 1)]):
        assert err(first + extra) > 1e-6 > 30 * six, extra
    fJ, gJ, eJ = _fp16_two_slice(J)
    fX, gX, eX = _fp16_two_slice(Xs)
    fp16 = (fJ @ fX.T + fJ @ gX.T + gJ @ fX.T) * 2.0 ** (-eJ) * 2.0 ** (-eX.T)
    assert np.linalg.norm(fp16 - exact) / np.linalg.norm(exact) < 3e-7
