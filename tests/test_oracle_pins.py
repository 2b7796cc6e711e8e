"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, textbook algorithms, library transforms, brute force, invariants).

None of these compare the oracle with itself: each check would fail on a plausible
mistake (dropped face, wrong sign, transposed axis, wrong window, wrong normalisation).
"""
import math
import os

import numpy as np
import pytest

from oracle import fcgno_oracle as O
from paper_2402_05598_gb300 import inputs as I

import closed_forms as CF


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------------------- stencil (Eq. 1-2)
@pytest.mark.parametrize("N", [3, 5, 8])
def test_stencil_equals_dense_matrix(N):
    rng = np.random.default_rng(N)
    k = I.grf_coefficient(N, rng, sigma=1.0, ell=0.2)
    A = O.dense_A(k)
    u = rng.standard_normal((N, N))
    assert rel(O.apply_A(k, u).ravel(), A @ u.ravel()) < 1e-14


@pytest.mark.parametrize("N,axis,j", [(12, 1, 2), (12, 0, 3), (31, 1, 5), (9, 0, 1)])
def test_layered_coefficient_flux_balance_pins_harmonic_faces(N, axis, j):
    """Harmonic-mean faces and the boundary-face convention (Eq. (2), finite volumes), pinned
    without restating the formula: on a coefficient layered along one axis, a grid function
    that carries a constant flux through series half-cell resistances has a closed-form
    A u at every node (tests/closed_forms.py). An arithmetic-mean face, a boundary face with
    a halved or doubled coefficient, a missing 1/h^2, or k taken from the wrong neighbour on
    the cross faces each breaks the balance."""
    k, u, Au = CF.layered_flux_field(N, axis=axis, j=j, seed=N + axis)
    got = O.apply_A(k, u)
    assert np.max(np.abs(got - Au)) <= 1e-12 * np.max(np.abs(Au))
    # the dense matrix (assembled separately, row by row) obeys the same balance
    assert np.max(np.abs((O.dense_A(k) @ u.ravel()).reshape(N, N) - Au)) <= 1e-12 * np.max(np.abs(Au))


def test_layered_flux_balance_rejects_an_arithmetic_mean_face(monkeypatch):
    """The layered-field pin has teeth: the same oracle with the arithmetic mean planted in
    place of the harmonic one fails it (at every node next to a face between unequal k)."""
    k, u, Au = CF.layered_flux_field(12, axis=1, j=2, seed=13)
    monkeypatch.setattr(O, "_harmonic", lambda a, b: 0.5 * (a + b))
    got = O.apply_A(k, u)
    assert np.max(np.abs(got - Au)) > 1e-3 * np.max(np.abs(Au))


@pytest.mark.parametrize("N", [4, 7])
def test_dense_matrix_symmetric_positive_definite(N):
    rng = np.random.default_rng(10 + N)
    k = I.grf_coefficient(N, rng, sigma=2.0, ell=0.1)
    A = O.dense_A(k)
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    np.linalg.cholesky(A)  # raises if not SPD
    # five-point structure: at most 5 nonzeros per row, off-diagonals negative
    assert np.all((A != 0).sum(axis=1) <= 5)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)


def test_constant_k_row_sums_are_boundary_faces():
    N, c = 6, 3.0
    A = O.dense_A(np.full((N, N), c))
    h = 1.0 / (N + 1)
    rs = A.sum(axis=1).reshape(N, N)
    expect = np.zeros((N, N))
    expect[:, 0] += c
    expect[:, -1] += c
    expect[0, :] += c
    expect[-1, :] += c
    assert np.allclose(rs, expect / h**2, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("N,i,j", [(16, 1, 1), (16, 3, 7), (33, 5, 2)])
def test_sine_eigenmode_closed_form(N, i, j):
    """Constant k = c and f = sin(i pi x) sin(j pi y): A f = c lambda f with
    lambda = (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)); the FCG(B=I) solve returns f/(c lambda)."""
    c = 2.5
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    f = np.outer(np.sin(j * np.pi * x), np.sin(i * np.pi * x))  # [q][p]: x2 mode j, x1 mode i
    lam = 4.0 / h**2 * (np.sin(i * np.pi * h / 2) ** 2 + np.sin(j * np.pi * h / 2) ** 2)
    k = np.full((N, N), c)
    assert rel(O.apply_A(k, f), c * lam * f) < 1e-12
    out = O.fcg(lambda u: O.apply_A(k, u), lambda r: r, f, np.zeros_like(f), 1, 10, tol=1e-14)
    assert rel(out["u"], f / (c * lam)) < 1e-12


# --------------------------------------------------------------------------- FCG (Algorithm 1)
def test_truncation_window_rule():
    # m_i = min(i, max(1, i mod (m_max+1)))
    assert [O.truncation_window(i, 1) for i in range(6)] == [0, 1, 1, 1, 1, 1]
    assert [O.truncation_window(i, 5) for i in range(14)] == [0, 1, 2, 3, 4, 5, 1, 1, 2, 3, 4, 5, 1, 1]


def test_fcg_identity_equals_textbook_cg():
    N = 12
    k, f = I.make_problem(N, 7)
    A = lambda u: O.apply_A(k, u)
    u0 = np.random.default_rng(1).standard_normal((N, N))
    a = O.fcg(A, lambda r: r, f, u0, 1, 10, record=True)
    b = O.cg_textbook(A, f, u0, 10)
    # the two recurrences round differently; on early iterations they agree to ~1e-13
    for i in range(1, 11):
        assert rel(a["us"][i], b["us"][i]) < 1e-11, i


@pytest.mark.parametrize("N", [4, 8])
def test_cg_finite_termination_matches_dense_solve(N):
    """n <= 64: CG terminates at the dense LU solution (1e-12). In exact arithmetic that takes
    at most n iterations; rounding delays it by a few (textbook CG shows the same delay)."""
    k, f = I.make_problem(N, 3)
    A = O.dense_A(k)
    u_lu = np.linalg.solve(A, f.ravel()).reshape(N, N)
    n = N * N
    out = O.fcg(lambda u: O.apply_A(k, u), lambda r: r, f, np.zeros_like(f), 1, n + n // 4 + 2, tol=1e-15)
    assert rel(out["u"], u_lu) < 1e-12
    ref = O.cg_textbook(lambda u: O.apply_A(k, u), f, np.zeros_like(f), out["iterations"])
    assert rel(ref["u"], u_lu) < 1e-12


def test_fcg_full_window_linear_preconditioner_equals_pcg():
    """With a fixed SPD linear B and m_max >= iters, FCG is PCG with that preconditioner."""
    N = 10
    k, f = I.make_problem(N, 11)
    A = lambda u: O.apply_A(k, u)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((N * N, N * N))
    Mi = G @ G.T / (N * N) + np.eye(N * N)
    B = lambda r: (Mi @ r.ravel()).reshape(N, N)
    u0 = rng.standard_normal((N, N))
    a = O.fcg(A, B, f, u0, 8, 8, record=True)
    b = O.pcg_textbook(A, B, f, u0, 8)
    for i in range(1, 9):
        assert rel(a["us"][i], b["us"][i]) < 1e-8, i


def test_fcg_energy_error_monotone_and_window_orthogonality_with_neural_preconditioner():
    """Exact line search: ||u* - u_i||_A never increases; p_i is A-orthogonal to the window."""
    N = 16
    desc = I.ModelDesc(width=8, layers=2, modes=4, proj_width=8)
    P = O.unpack_weights(I.xavier_weights(desc, 3), desc)
    k, f = I.make_problem(N, 5)
    A = lambda u: O.apply_A(k, u)
    ustar = np.linalg.solve(O.dense_A(k), f.ravel()).reshape(N, N)
    m_max = 3
    out = O.fcg(A, lambda r: O.no_forward(P, desc, r, np.log(k)), f, np.zeros_like(f), m_max, 20, record=True)
    errs = [O.energy_norm(k, ustar - u) for u in out["us"]]
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
    ps, ss = out["ps"], out["ss"]
    for i in range(1, len(ps)):
        for kk in range(i - O.truncation_window(i, m_max), i):
            assert abs(np.sum(ps[i] * ss[kk])) <= 1e-9 * math.sqrt(np.sum(ps[i] * A(ps[i])) * np.sum(ps[kk] * ss[kk]))


def test_fcg_recursive_residual_is_the_true_residual():
    """Algorithm 1 updates r by r - alpha A p instead of recomputing f - A u: in exact
    arithmetic the two agree at every iteration, in FP64 they drift only by rounding. A sign
    or index slip in either update makes them part at the first iteration."""
    N = 16
    desc = I.ModelDesc(width=8, layers=2, modes=4, proj_width=8)
    P = O.unpack_weights(I.xavier_weights(desc, 4), desc)
    k, f = I.make_problem(N, 6)
    A = lambda u: O.apply_A(k, u)
    u0 = np.random.default_rng(7).standard_normal((N, N))
    for m_max in (1, 5):
        out = O.fcg(A, lambda r: O.no_forward(P, desc, r, np.log(k)), f, u0, m_max, 30, record=True)
        assert out["iterations"] == 30
        for u, r in zip(out["us"], out["rs"]):
            assert np.linalg.norm(r - (f - A(u))) <= 1e-11 * out["r0"]
        # the untrained preconditioner barely lowers the residual, but the iterate moves
        assert np.linalg.norm(out["u"] - u0) >= 0.1 * np.linalg.norm(u0)


def test_fcg_step_is_an_exact_line_search():
    """alpha = (p_i, r_i) / (p_i, A p_i) minimises the energy error along p_i, so the new
    residual is orthogonal to the search direction: (p_i, r_{i+1}) = 0 at every iteration,
    also with a nonlinear preconditioner and a truncated window; and p_i is A-orthogonal to
    the window it was orthogonalised against."""
    N = 12
    desc = I.ModelDesc(width=8, layers=2, modes=3, proj_width=8)
    P = O.unpack_weights(I.xavier_weights(desc, 9), desc)
    k, f = I.make_problem(N, 13)
    A = lambda u: O.apply_A(k, u)
    for m_max in (1, 3, 5):
        out = O.fcg(A, lambda r: O.no_forward(P, desc, r, np.log(k)), f, np.zeros_like(f), m_max, 25,
                    record=True)
        ps, rs = out["ps"], out["rs"]
        for i, p in enumerate(ps):
            rn = rs[i + 1]
            assert abs(np.sum(p * rn)) <= 1e-10 * np.linalg.norm(p) * np.linalg.norm(rs[i])
            for kk in range(i - O.truncation_window(i, m_max), i):
                Ap = A(ps[kk])
                assert abs(np.sum(p * Ap)) <= 1e-9 * math.sqrt(np.sum(p * A(p)) * np.sum(ps[kk] * Ap))


def table1():
    """Rows (dataset, grid, CG iterations, Jacobi(4) iterations) of Table 1, from
    tests/golden/table1_iterations.txt."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_iterations.txt")
    rows = []
    with open(path) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                ds, grid, cg, jac = ln.split()
                rows.append((ds, int(grid), int(cg), int(jac)))
    return rows


GENERATORS = {"poisson": I.poisson_problem, "diffusion": I.diffusion_problem}


def test_table1_cg_iteration_counts_soft_pin():
    """Table 1: the iterations CG needs to reach ||r_i||/||r_0|| <= 1e-6 from u_0 ~ N(0, 1) on
    the Poisson and Diffusion datasets at grids 32, 64 and 128. Soft pin (+-15%): the paper's
    grid convention and draws are not published."""
    rows = table1()
    assert len(rows) == 6
    for ds, N, target, _ in rows:
        its = []
        for s in range(3):
            k, f = GENERATORS[ds](N, s)
            u0 = np.random.default_rng(100 + s).standard_normal((N, N))
            its.append(O.fcg(lambda u: O.apply_A(k, u), lambda r: r, f, u0, 1, 1000, tol=1e-6)["iterations"])
        assert abs(np.mean(its) - target) <= 0.15 * target, (N, ds, its)


def test_jacobi_preconditioner_fixed_point_and_steps():
    """Eq. (15): Jacobi(k) from x0 = 0; one step is D^-1 r, and many steps converge to A^-1 r
    (the FV matrix is weakly diagonally dominant and irreducible)."""
    N = 6
    k, r = I.make_problem(N, 4)
    A = O.dense_A(k)
    d = np.diag(A).reshape(N, N)
    assert rel(O.jacobi_precond(k, r, 1), r / d) < 1e-15
    x = O.jacobi_precond(k, r, 3000)
    assert rel(x.ravel(), np.linalg.solve(A, r.ravel())) < 1e-8


# --------------------------------------------------------------------------- truncated DFT
@pytest.mark.parametrize("N,M", [(16, 4), (20, 5), (32, 8)])
def test_analysis_matches_numpy_fft(N, M):
    rng = np.random.default_rng(N)
    v = rng.standard_normal((N, N, 3))
    c = O.analysis(v, M)
    F = np.fft.fft2(v, axes=(0, 1)) / (N * N)   # F[k2][k1] over axes (q, p)
    k1 = O.kx_frequencies(M) % N
    ref = np.transpose(F[:M][:, k1], (1, 0, 2))  # -> [k1 slot][k2][C]
    assert np.max(np.abs(c - ref)) < 1e-13


def test_single_mode_is_one_hot():
    N, M = 16, 4
    p = np.arange(N)[None, :]
    q = np.arange(N)[:, None]
    k1, k2 = -3, 2
    v = np.cos(2 * np.pi * (k1 * p + k2 * q) / N)[..., None]
    c = O.analysis(v, M)
    j = list(O.kx_frequencies(M)).index(k1)
    expect = np.zeros_like(c)
    expect[j, k2, 0] = 0.5  # cos = (e^{i t} + e^{-i t}) / 2; the mirror has k2 = -2, not kept
    assert np.max(np.abs(c - expect)) < 1e-14


def _band_limited(N, M, rng, C=2):
    p = np.arange(N)[None, :, None]
    q = np.arange(N)[:, None, None]
    v = np.zeros((N, N, C))
    for k1 in range(-(M - 1), M):
        for k2 in range(M):
            a = rng.standard_normal(C) + 1j * rng.standard_normal(C)
            v += np.real(a * np.exp(2j * np.pi * (k1 * p + k2 * q) / N))
    return v


@pytest.mark.parametrize("N,M", [(16, 4), (24, 6), (12, 6)])
def test_synthesis_inverts_analysis_on_band_limited_fields(N, M):
    v = _band_limited(N, M, np.random.default_rng(M))
    assert rel(O.synthesis(O.analysis(v, M), N), v) < 1e-13


def test_resolution_consistency_of_coefficients():
    """The same band-limited function sampled on N and 2N points has equal coefficients."""
    M = 4
    rng = np.random.default_rng(0)
    coef = {(k1, k2): rng.standard_normal() + 1j * rng.standard_normal() for k1 in range(-(M - 1), M) for k2 in range(M)}

    def sample(N):
        x = np.arange(N) / N
        v = np.zeros((N, N, 1))
        for (k1, k2), a in coef.items():
            v[..., 0] += np.real(a * np.exp(2j * np.pi * (k1 * x[None, :] + k2 * x[:, None])))
        return v

    assert np.max(np.abs(O.analysis(sample(16), M) - O.analysis(sample(32), M))) < 1e-13


def test_mode_mix_phase_rotation_shifts_plane_wave():
    """R(k) = exp(-i k1 2 pi s / N) I shifts every retained plane wave by s in x1."""
    N, M, C, s = 16, 4, 2, 3
    v = _band_limited(N, M, np.random.default_rng(5), C)
    k1 = O.kx_frequencies(M)
    R = np.zeros((2 * M, M, C, C), dtype=complex)
    for j in range(2 * M):
        R[j, :, :, :] = np.exp(-2j * np.pi * k1[j] * s / N) * np.eye(C)
    out = O.synthesis(O.mode_mix(O.analysis(v, M), R), N)
    assert rel(out, np.roll(v, s, axis=1)) < 1e-13


def test_gelu_values():
    assert abs(O.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(O.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    assert O.gelu(np.array([0.0]))[0] == 0.0


def test_fourier_layer_identity_reproduces_band_limited_input():
    N, M, C = 16, 4, 3
    v = _band_limited(N, M, np.random.default_rng(9), C)
    layer = {"w": np.zeros((C, C)), "b": np.zeros(C), "r": np.broadcast_to(np.eye(C), (2 * M, M, C, C)).astype(complex)}
    assert rel(O.fourier_layer(v, layer, M, activate=False), v) < 1e-13
    # pointwise path alone: R = 0 gives W v + b
    W = np.random.default_rng(1).standard_normal((C, C))
    b = np.arange(C, dtype=float)
    layer2 = {"w": W, "b": b, "r": np.zeros((2 * M, M, C, C), dtype=complex)}
    assert rel(O.fourier_layer(v, layer2, M, activate=False), v @ W.T + b) < 1e-14


# --------------------------------------------------------------------------- full NO invariants
def _model(C=8, M=4, L=3, seed=0):
    desc = I.ModelDesc(width=C, layers=L, modes=M, proj_width=C)
    return desc, O.unpack_weights(I.xavier_weights(desc, seed), desc)


def test_no_shift_equivariance_and_homogeneity():
    N = 16
    desc, P = _model()
    k, r = I.make_problem(N, 2)
    lk = np.log(k)
    z = O.no_forward(P, desc, r, lk)
    zs = O.no_forward(P, desc, np.roll(r, (3, 5), axis=(0, 1)), np.roll(lk, (3, 5), axis=(0, 1)))
    assert rel(zs, np.roll(z, (3, 5), axis=(0, 1))) < 1e-12
    assert rel(O.no_forward(P, desc, 7.5 * r, lk), 7.5 * z) < 1e-13
    assert np.all(O.no_forward(P, desc, np.zeros_like(r), lk) == 0)


def test_weight_blob_layout_and_xavier_bounds():
    desc = I.ModelDesc(width=16, layers=4, modes=8, proj_width=16)
    blob = I.xavier_weights(desc, 0)
    C, M = 16, 8
    expect = C * 2 + C + 4 * (C * C + C + 2 * M * M * C * C * 2) + C * C + C + C + 1
    assert blob.size == expect == I.weight_count(desc)
    P = O.unpack_weights(blob, desc)
    assert np.all(np.abs(P["layers"][0]["w"]) <= math.sqrt(6 / (2 * C)))
    assert np.all(np.abs(P["layers"][0]["r"].real) <= math.sqrt(6 / (2 * C)))
    assert np.all(P["layers"][2]["b"] == 0)


# --------------------------------------------------------------------------- losses (Eq. 11-12)
@pytest.mark.parametrize("out_scale", [0, 1])
def test_pointwise_no_reduces_to_a_scalar_closed_form(out_scale):
    """With every spectral block R_l = 0 and W_l = I the Fourier layers act node by node, so
    the whole preconditioner of Appendix A reduces to a scalar function of (r/rms, log k) at
    each node: encoder a r^ + b log k + c, GELU(u + b_l) on layers 1-3, u + b_4 on the last,
    decoder s . GELU(P u + q) + t, times h^2 rms(r) (and divided by the node's k for
    output_scale 1). Computed here node by node with math.erf and math.exp, it pins the
    encoder's channel order, which layers apply GELU, the biases, the decoder and the output
    scale with h = 1/(N+1)."""
    N, C, Cp, L, M = 8, 4, 3, 4, 2
    desc = I.ModelDesc(width=C, layers=L, modes=M, proj_width=Cp, output_scale=out_scale)
    off = I.weight_offsets(desc)
    blob = np.zeros(I.weight_count(desc), dtype=np.float32)
    rng = np.random.default_rng(11)

    def put(name, values):
        o, size = off[name]
        values = np.asarray(values, dtype=np.float32).ravel()
        assert values.size == size
        blob[o:o + size] = values

    lift_w = rng.uniform(-1, 1, (C, 2))
    lift_b = rng.uniform(-0.5, 0.5, C)
    put("lift_w", lift_w)
    put("lift_b", lift_b)
    biases = [rng.uniform(-0.5, 0.5, C) for _ in range(L)]
    for l in range(L):
        put(f"w{l}", np.eye(C))
        put(f"b{l}", biases[l])
    P1 = rng.uniform(-1, 1, (Cp, C))
    q = rng.uniform(-0.5, 0.5, Cp)
    s2 = rng.uniform(-1, 1, Cp)
    t = 0.3
    put("proj1_w", P1)
    put("proj1_b", q)
    put("proj2_w", s2)
    put("proj2_b", [t])
    # read the parameters back as the stored float32 values
    lift_w, lift_b = blob[off["lift_w"][0]:][:C * 2].reshape(C, 2).astype(float), blob[off["lift_b"][0]:][:C]
    biases = [blob[off[f"b{l}"][0]:][:C].astype(float) for l in range(L)]
    P1 = blob[off["proj1_w"][0]:][:Cp * C].reshape(Cp, C).astype(float)
    q, s2 = blob[off["proj1_b"][0]:][:Cp].astype(float), blob[off["proj2_w"][0]:][:Cp].astype(float)
    t = float(blob[off["proj2_b"][0]])

    def g(x):
        return 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))

    r = rng.standard_normal((N, N))
    logk = rng.uniform(-1, 1, (N, N))
    z = O.no_forward(O.unpack_weights(blob, desc), desc, r, logk)
    rms = math.sqrt(sum(v * v for v in r.ravel()) / (N * N))
    h = 1.0 / (N + 1)
    for qq in range(N):
        for pp in range(N):
            u = [lift_w[c][0] * r[qq, pp] / rms + lift_w[c][1] * logk[qq, pp] + float(lift_b[c]) for c in range(C)]
            for l in range(L):
                u = [u[c] + biases[l][c] for c in range(C)]
                if l < L - 1:
                    u = [g(x) for x in u]
            hid = [g(sum(P1[j][c] * u[c] for c in range(C)) + q[j]) for j in range(Cp)]
            want = h * h * rms * (sum(s2[j] * hid[j] for j in range(Cp)) + t)
            if out_scale:
                want /= math.exp(logk[qq, pp])
            assert abs(z[qq, pp] - want) <= 1e-12 * max(1.0, abs(want)) * h * h, (qq, pp, z[qq, pp], want)


def test_spectral_weight_layout_single_mode_closed_form():
    """The documented layout of the spectral weights r_l [2M][M][C][C][2] (x1 slot j holds
    frequency j or j - 2M, then the x2 frequency, input channel, output channel, re/im) and the
    transform conventions, end to end through a one-layer NO. Input r = cos(theta) with
    theta = 2 pi (k1 p + k2 q) / N, k1 = -2 (slot 2M - 2), k2 = 1; the encoder copies r/rms
    into channel 0; the only nonzero spectral weight is R[slot, k2, in 0, out 1] = alpha +
    i beta; the decoder reads channel 1 through one GELU. The kept coefficient of
    r/rms = sqrt(2) cos(theta) is sqrt(2)/2 at (k1, k2) (its mirror has x2-frequency -1, which
    is not kept) and synthesis doubles k2 > 0 terms, so
    z = h^2 rms(r) GELU(sqrt(2) (alpha cos(theta) - beta sin(theta))). The same weight placed
    at (in 1, out 0) reads the empty channel and gives z = 0."""
    N, C, Cp, L, M = 8, 2, 2, 1, 3
    k1, k2 = -2, 1
    slot = k1 + 2 * M
    assert O.kx_frequencies(M)[slot] == k1
    alpha, beta = 0.7, -0.4
    desc = I.ModelDesc(width=C, layers=L, modes=M, proj_width=Cp)
    off = I.weight_offsets(desc)

    def blob_with(cin, cout):
        blob = np.zeros(I.weight_count(desc), dtype=np.float64)
        blob[off["lift_w"][0] + 0] = 1.0               # lift_w[0][0]: r/rms -> channel 0
        base = off["r0"][0] + ((((slot * M + k2) * C + cin) * C + cout) * 2)
        blob[base], blob[base + 1] = alpha, beta
        blob[off["proj1_w"][0] + 0 * C + 1] = 1.0      # proj1_w[0][1]: channel 1 -> hidden 0
        blob[off["proj2_w"][0] + 0] = 1.0              # proj2_w[0]
        return blob

    rng = np.random.default_rng(5)
    pp, qq = np.meshgrid(np.arange(N), np.arange(N))   # arrays indexed [q][p]
    theta = 2 * np.pi * (k1 * pp + k2 * qq) / N
    r = np.cos(theta)
    logk = rng.uniform(-1, 1, (N, N))
    h = 1.0 / (N + 1)
    rms = math.sqrt(0.5)
    z = O.no_forward(O.unpack_weights(blob_with(0, 1), desc), desc, r, logk)
    for q_ in range(N):
        for p_ in range(N):
            x = math.sqrt(2.0) * (alpha * math.cos(theta[q_, p_]) - beta * math.sin(theta[q_, p_]))
            want = h * h * rms * 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))
            assert abs(z[q_, p_] - want) <= 1e-13 * h * h, (q_, p_, z[q_, p_], want)
    z0 = O.no_forward(O.unpack_weights(blob_with(1, 0), desc), desc, r, logk)
    assert np.max(np.abs(z0)) <= 1e-15


def test_constant_fields_follow_the_mean_mode_through_every_layer():
    """For constant r and log k every channel stays constant through the whole NO, so only
    the mean mode (k1, k2) = (0, 0) is nonzero: each Fourier layer maps the channel vector u
    to act(W u + b + Re(R_00)^T u) (the mode's synthesis weight is 1 and only the real part
    of its complex weight acts), with all other weights random and irrelevant. Computed here
    by scalar loops through all four layers, GELU on the first three, and the decoder."""
    N, C, Cp, L, M = 8, 3, 2, 4, 3
    desc = I.ModelDesc(width=C, layers=L, modes=M, proj_width=Cp)
    blob = I.xavier_weights(desc, 21).astype(np.float64)
    rng = np.random.default_rng(2)
    off = I.weight_offsets(desc)
    for l in range(L):  # nonzero biases so that they are exercised too
        o, size = off[f"b{l}"]
        blob[o:o + size] = rng.uniform(-0.3, 0.3, size)
    P = O.unpack_weights(blob, desc)
    cr, lk = -0.8, 0.35
    r = np.full((N, N), cr)
    logk = np.full((N, N), lk)
    z = O.no_forward(P, desc, r, logk)

    def g(x):
        return 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0)))

    lw, lb = P["lift_w"], P["lift_b"]
    u = [lw[c][0] * (cr / abs(cr)) + lw[c][1] * lk + lb[c] for c in range(C)]
    for l, lay in enumerate(P["layers"]):
        W, b, R00 = lay["w"], lay["b"], lay["r"][0, 0]
        u = [sum(W[o][i] * u[i] for i in range(C)) + b[o] + sum(R00[i][o].real * u[i] for i in range(C))
             for o in range(C)]
        if l < L - 1:
            u = [g(x) for x in u]
    hid = [g(sum(P["proj1_w"][j][c] * u[c] for c in range(C)) + P["proj1_b"][j]) for j in range(Cp)]
    h = 1.0 / (N + 1)
    want = h * h * abs(cr) * (sum(P["proj2_w"][j] * hid[j] for j in range(Cp)) + P["proj2_b"][0])
    assert np.max(np.abs(z - want)) <= 1e-12 * h * h * max(1.0, abs(want) / (h * h))


def _no_by_full_grid_fft(P, desc, r, logk):
    """The neural operator stated a second way, for the pin below: each spectral layer takes the
    whole grid's discrete Fourier transform with numpy's FFT, picks the kept modes out of it,
    mixes them, places the mixed coefficients (doubled for x2-frequencies above 0) into an
    otherwise empty N x N spectrum and returns the real part of numpy's inverse FFT, instead of
    the oracle's dense truncated twiddle products. GELU comes from math.erf, the pointwise maps
    are explicit loops over channels."""
    N, C, M = r.shape[0], desc.width, desc.modes
    n = N * N
    gelu = np.vectorize(lambda x: 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0))))
    rms = math.sqrt(float(np.sum(r * r)) / n)
    x_in = [r / rms, logk]
    v = np.stack([sum(P["lift_w"][c][i] * x_in[i] for i in range(2)) + P["lift_b"][c] for c in range(C)], axis=-1)
    k1_of_slot = list(range(M)) + list(range(-M, 0))
    L = len(P["layers"])
    for l, lay in enumerate(P["layers"]):
        spec_in = np.fft.fft2(v, axes=(0, 1)) / n          # [x2 frequency][x1 frequency][channel]
        full = np.zeros((N, N, C), dtype=complex)
        for j, k1 in enumerate(k1_of_slot):
            for k2 in range(M):
                cin = spec_in[k2, k1 % N, :]
                cout = np.array([sum(cin[i] * lay["r"][j, k2, i, o] for i in range(C)) for o in range(C)])
                full[k2, k1 % N, :] += (1.0 if k2 == 0 else 2.0) * cout
        spec = np.real(np.fft.ifft2(full, axes=(0, 1))) * n
        h = np.stack([sum(lay["w"][o][i] * v[..., i] for i in range(C)) + lay["b"][o] for o in range(C)], axis=-1)
        h = h + spec
        v = gelu(h) if l < L - 1 else h
    Cp = desc.proj_width
    hid = [gelu(sum(P["proj1_w"][j][c] * v[..., c] for c in range(C)) + P["proj1_b"][j]) for j in range(Cp)]
    zt = sum(P["proj2_w"][j] * hid[j] for j in range(Cp)) + P["proj2_b"][0]
    scale = (1.0 / (N + 1)) ** 2 * rms
    if desc.output_scale:
        scale = scale * np.exp(-logk)
    return scale * zt


@pytest.mark.parametrize("N,C,M,out_scale", [(16, 4, 4, 0), (12, 3, 5, 1), (20, 4, 3, 1)])
def test_composed_no_with_random_weights_matches_a_full_grid_fft_statement(N, C, M, out_scale):
    """The whole four-layer neural operator with random weights in every block (encoder, W_l,
    b_l, all 2M x M spectral blocks, decoder) against the second statement above, which reaches
    the kept modes through full-grid FFTs: a slip anywhere in the oracle's truncated transforms,
    their slot order, the mixing's index order, the synthesis weights, the layer composition or
    the output scale that the one-mode and constant-field pins leave open shows up here with all
    modes active at once. N = 12 and 20 are not powers of two; at N = 12, M = 5 the x1
    frequencies -5..4 nearly fill the grid."""
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C, output_scale=out_scale)
    blob = I.xavier_weights(desc, 40 + N).astype(np.float64)
    rng = np.random.default_rng(N)
    off = I.weight_offsets(desc)
    for name in ["lift_b", "proj1_b", "proj2_b"] + [f"b{l}" for l in range(4)]:
        o, size = off[name]
        blob[o:o + size] = rng.uniform(-0.3, 0.3, size)
    P = O.unpack_weights(blob, desc)
    k, r = I.make_problem(N, 7 + N)
    logk = np.log(k)
    z = O.no_forward(P, desc, r, logk)
    want = _no_by_full_grid_fft(P, desc, r, logk)
    assert rel(z, want) < 1e-12
    assert np.max(np.abs(z - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("slip", ["mixing transposed", "conjugated weights", "x1 slots reversed",
                                  "grid axes swapped"])
def test_full_grid_fft_statement_rejects_planted_slips(monkeypatch, slip):
    """The pin above fails when a plausible slip is planted in the oracle: the mixing's
    input/output indices exchanged, the spectral weights conjugated, the negative x1 frequencies
    stored in reverse slot order, or the analysis taken over the grid's axes exchanged."""
    mix, kx, ana = O.mode_mix, O.kx_frequencies, O.analysis
    if slip == "mixing transposed":
        monkeypatch.setattr(O, "mode_mix", lambda c, R: mix(c, np.swapaxes(R, 2, 3)))
    elif slip == "conjugated weights":
        monkeypatch.setattr(O, "mode_mix", lambda c, R: mix(c, np.conj(R)))
    elif slip == "x1 slots reversed":
        monkeypatch.setattr(O, "kx_frequencies", lambda M: np.concatenate([np.arange(M), -np.arange(1, M + 1)]))
    else:
        monkeypatch.setattr(O, "analysis", lambda v, M: ana(np.swapaxes(v, 0, 1), M))
    with pytest.raises(AssertionError):
        test_composed_no_with_random_weights_matches_a_full_grid_fft_statement(16, 4, 4, 0)


def test_notay_loss_exact_inverse_is_zero_and_zero_output_is_one():
    N = 6
    k, r = I.make_problem(N, 8)
    e = np.linalg.solve(O.dense_A(k), r.ravel()).reshape(N, N)
    assert O.notay_loss([k], [e.copy()], [e]) < 1e-12
    assert abs(O.notay_loss([k], [np.zeros_like(e)], [e]) - 1.0) < 1e-15
    assert abs(O.l2_loss([np.zeros_like(e)], [e]) - 1.0) < 1e-15


def test_losses_are_batch_means_of_norm_ratios():
    """Eq. (11) as read: the batch mean of ||z - e||_A / ||e||_A, a ratio of norms and not of
    squared norms (z = e/2 gives 1/2, not 1/4), averaged and not summed (an exact and a zero
    output give 1/2, not 1); the L2 ablation loss the same with the Euclidean norm. Both are
    invariant to a common scale of z and e."""
    N = 6
    k1, r1 = I.make_problem(N, 8)
    k2, r2 = I.make_problem(N, 9)
    e1 = np.linalg.solve(O.dense_A(k1), r1.ravel()).reshape(N, N)
    e2 = np.linalg.solve(O.dense_A(k2), r2.ravel()).reshape(N, N)
    assert abs(O.notay_loss([k1], [0.5 * e1], [e1]) - 0.5) < 1e-14
    assert abs(O.l2_loss([0.5 * e1], [e1]) - 0.5) < 1e-14
    assert abs(O.notay_loss([k1, k2], [e1.copy(), np.zeros_like(e2)], [e1, e2]) - 0.5) < 1e-12
    assert abs(O.l2_loss([e1.copy(), np.zeros_like(e2)], [e1, e2]) - 0.5) < 1e-12
    z1 = e1 + 0.1 * np.random.default_rng(1).standard_normal(e1.shape)
    assert abs(O.notay_loss([k1], [3.0 * z1], [3.0 * e1]) - O.notay_loss([k1], [z1], [e1])) < 1e-13
    assert abs(O.l2_loss([3.0 * z1], [3.0 * e1]) - O.l2_loss([z1], [e1])) < 1e-13


# --------------------------------------------------------------------------- inputs
def test_grf_sample_covariance():
    """Statistical check of the GRF generator: empirical covariance of g = log k between
    nodes at distance d approaches sigma^2 exp(-d^2 / (2 l^2))."""
    N, sigma, ell = 12, 1.3, 0.15
    rng = np.random.default_rng(0)
    g = np.stack([np.log(I.grf_coefficient(N, rng, sigma, ell)) for _ in range(3000)])
    h = 1.0 / (N + 1)
    for dp in (0, 1, 3):
        emp = np.mean(g[:, 5, 4] * g[:, 5, 4 + dp])
        assert abs(emp - sigma**2 * math.exp(-((dp * h) ** 2) / (2 * ell**2))) < 0.12 * sigma**2


# --------------------------------------------------------------------------- training gradient
def test_transform_adjoints_by_inner_products():
    """<S c, g> = <c, S^T g> and <A v, d> = <v, A^T d> with complex inputs read as (re, im)."""
    N, M, C = 12, 3, 2
    rng = np.random.default_rng(4)
    c = rng.standard_normal((2 * M, M, C)) + 1j * rng.standard_normal((2 * M, M, C))
    g = rng.standard_normal((N, N, C))
    lhs = np.sum(O.synthesis(c, N) * g)
    adj = O.synthesis_adjoint(g, M)
    rhs = np.sum(c.real * adj.real + c.imag * adj.imag)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    v = rng.standard_normal((N, N, C))
    d = rng.standard_normal((2 * M, M, C)) + 1j * rng.standard_normal((2 * M, M, C))
    a = O.analysis(v, M)
    lhs = np.sum(a.real * d.real + a.imag * d.imag)
    rhs = np.sum(v * O.analysis_adjoint(d, N))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("kind", ["energy", "l2"])
@pytest.mark.parametrize("out_scale", [0, 1])
def test_loss_gradient_matches_central_differences(kind, out_scale):
    """The hand-written reverse mode of Eq. (11) (energy) and of the L2 ablation loss against
    central finite differences on every parameter group (random coordinates), FP64,
    agreement to 1e-6 relative, for both output scales; the loss value equals the separately
    written loss."""
    N = 10
    desc = I.ModelDesc(width=4, layers=2, modes=3, proj_width=4, output_scale=out_scale)
    blob = I.xavier_weights(desc, 1).astype(np.float64)
    off = I.weight_offsets(desc)
    rng = np.random.default_rng(0)
    for name in ["lift_b", "proj1_b", "proj2_b", "b0", "b1"]:
        o, s = off[name]
        blob[o:o + s] = rng.uniform(-0.3, 0.3, s)
    ks, rs, es = [], [], []
    for s in range(2):
        k, f = I.make_problem(N, 40 + s)
        e = np.linalg.solve(O.dense_A(k), f.ravel()).reshape(N, N)
        ks.append(k)
        rs.append(f)
        es.append(e)
    fn = O.notay_loss_and_grad if kind == "energy" else O.l2_loss_and_grad

    def loss_of(b):
        return fn(O.unpack_weights(b, desc), desc, ks, rs, es)[0]

    L0, g = fn(O.unpack_weights(blob, desc), desc, ks, rs, es)
    zs = [O.no_forward(O.unpack_weights(blob, desc), desc, r, np.log(k)) for k, r in zip(ks, rs)]
    direct = O.notay_loss(ks, zs, es) if kind == "energy" else O.l2_loss(zs, es)
    assert abs(L0 - direct) < 1e-14
    checked = 0
    for name, (o, s) in off.items():
        if name == "_total":
            continue
        for idx in rng.choice(s, size=min(s, 3), replace=False):
            i = o + idx
            h = 1e-6 * max(1.0, abs(blob[i]))
            bp = blob.copy()
            bm = blob.copy()
            bp[i] += h
            bm[i] -= h
            fd = (loss_of(bp) - loss_of(bm)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (name, idx, fd, g[i])
            checked += 1
    assert checked >= 20


def test_table1_jacobi4_iteration_counts_soft_pin():
    """Table 1: the iterations FCG with Jacobi(4) needs to reach 1e-6 from u_0 ~ N(0, 1) at
    grids 32, 64 and 128. Soft pin (+-20%)."""
    for ds, N, _, target in table1():
        its = []
        for s in range(2):
            k, f = GENERATORS[ds](N, s)
            u0 = np.random.default_rng(100 + s).standard_normal((N, N))
            out = O.fcg(lambda u: O.apply_A(k, u), lambda r: O.jacobi_precond(k, r, 4), f, u0, 1, 1000, tol=1e-6)
            its.append(out["iterations"])
        assert abs(np.mean(its) - target) <= 0.2 * target, (N, ds, its)
