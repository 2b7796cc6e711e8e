"""Plain FP64 CPU oracle of the FCG-NO method (Rudikov et al., arXiv 2402.05598).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module. It is deliberately slow and literal: every
function follows one passage of the paper (cited in its docstring) or a textbook
definition, with numpy primitives (matmul, einsum, erf, solve) as single steps and no
blocking, fusion or reordering beyond what the definition states. It shares no code with
the CUDA library.

Readings of points the paper leaves open (the same readings the library implements):
- Eq. (1) is read in divergence form, -div(k grad u) = f (the double sum over i, j is
  taken as i = j).
- Eq. (2) discretisation: N x N interior nodes, h = 1/(N+1), 5-point finite volume with
  harmonic-mean face coefficients 2 k_P k_Q / (k_P + k_Q); a face on the Dirichlet
  boundary takes k of its interior node; the operator carries the 1/h^2 scale. Arrays
  are [q][p] with p (the x1 index) fastest.
- Algorithm 1: u_0 is an explicit input; convergence is ||r_i|| <= tol ||r_0|| on the
  recursively updated residual (Table 1 caption); a zero or non-finite (p_i, s_i) stops
  the solve (breakdown), a zero residual counts as converged.
- Section 2.4.2 / Appendix A (neural operator): Fourier layers
  v <- act(W v + b + Re S R A v), act = GELU on all but the last layer, an encoder
  (lift, 2 -> C, linear) and a decoder (C -> C_p, GELU, -> 1) with C_p = C; the input
  channels are (r / rms(r), log k) and the output is rescaled by h^2 rms(r), so the map is
  positively homogeneous in r and returns 0 for r = 0. The h^2 factor gives the network
  output the units of A^-1 (A carries 1/h^2); FCG is invariant to a constant scale of w_i,
  so it only conditions the training loss, whose target e = A^-1 r is ~h^2 r at high
  frequencies. A model may also divide the output by k grid point by grid point
  (desc.output_scale = 1: z = h^2 rms(r) NO / k), the way k enters A^-1 ~ h^2 r / (4k) at
  the highest frequencies; the paper leaves the network's output scaling open.
- Retained modes: x1-frequencies 0..M-1 and -M..-1, x2-frequencies 0..M-1. Analysis
  c(k) = (1/n) sum_x v(x) exp(-2 pi i k.x / N), synthesis
  v(x) = Re sum_k w_k2 c(k) exp(+2 pi i k.x / N) with w_0 = 1, w_{k2>0} = 2.
- GELU is the exact erf form.

Pins (tests/test_oracle_pins.py) fix every component against closed forms, textbook
algorithms, numpy FFTs and the paper's Table 1. The composed neural-operator forward
(no_forward with random weights) has no closed form: its analysis, mixing, synthesis,
pointwise, GELU and encoder/decoder steps are each pinned, the whole map is checked for
shift equivariance and positive homogeneity, and with zero spectral blocks and identity W it
is checked node by node against a scalar closed form (encoder channel order, activations,
biases, decoder, the h^2 rms(r) scale); a one-layer NO with a single nonzero spectral weight
and a single-mode input is checked against its closed form (the weight layout and transform
conventions); constant inputs reduce the four-layer NO with random weights to its mean mode,
checked against scalar loops; with random weights in every block and non-constant inputs the
four-layer composition is checked against a second statement that reaches the kept modes
through numpy's full-grid FFTs and explicit channel loops (it shares this module's readings of
the paper, not its arithmetic; planted slips in the mixing, the slot order or the grid axes fail
it). FCG-NO iterates with such a preconditioner have no closed form; they are pinned through
properties Algorithm 1 guarantees for any preconditioner: monotone energy error, A-orthogonal
window directions, an exact line search and a recursively updated residual equal to f - A u.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

__all__ = [
    "grid_h",
    "face_coefficients",
    "apply_A",
    "dense_A",
    "truncation_window",
    "fcg",
    "cg_textbook",
    "pcg_textbook",
    "kx_frequencies",
    "analysis",
    "synthesis",
    "mode_mix",
    "gelu",
    "unpack_weights",
    "fourier_layer",
    "no_forward",
    "output_scale",
    "notay_loss",
    "l2_loss",
    "jacobi_precond",
    "energy_norm",
    "synthesis_adjoint",
    "analysis_adjoint",
    "gelu_grad",
    "notay_loss_and_grad",
]

STATUS_RUNNING = -1
STATUS_CONVERGED = 0
STATUS_MAXITER = 4
STATUS_BREAKDOWN = 5


# ---------------------------------------------------------------------------------------
# Discretisation (Section 2.1, Eq. (1)-(2))
# ---------------------------------------------------------------------------------------
def grid_h(N: int) -> float:
    """Mesh width of the N x N interior grid of the unit square (Eq. (1) domain (0,1)^2)."""
    return 1.0 / (N + 1)


def _harmonic(a, b):
    return 2.0 * a * b / (a + b)


def face_coefficients(k: np.ndarray):
    """Face coefficients of the 5-point finite-volume scheme for Eq. (1).

    Returns (aE, aW, aN, aS), each [N][N]: the coefficient on the east, west, north and
    south face of every interior node. Interior faces take the harmonic mean of the two
    nodes' k; boundary faces take the node's own k.
    """
    N = k.shape[0]
    aE = k.copy()
    aW = k.copy()
    aN = k.copy()
    aS = k.copy()
    aE[:, : N - 1] = _harmonic(k[:, : N - 1], k[:, 1:])
    aW[:, 1:] = _harmonic(k[:, 1:], k[:, : N - 1])
    aN[: N - 1, :] = _harmonic(k[: N - 1, :], k[1:, :])
    aS[1:, :] = _harmonic(k[1:, :], k[: N - 1, :])
    return aE, aW, aN, aS


def apply_A(k: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Matrix-free A u for the discretised Eq. (1) with zero Dirichlet data (Eq. (2)).

    (A u)_P = h^-2 [ (aE+aW+aN+aS) u_P - aE u_E - aW u_W - aN u_N - aS u_S ], with u = 0
    outside the interior grid.
    """
    N = k.shape[0]
    h = grid_h(N)
    aE, aW, aN, aS = face_coefficients(k)
    up = np.zeros((N + 2, N + 2))
    up[1:-1, 1:-1] = u
    uE = up[1:-1, 2:]
    uW = up[1:-1, :-2]
    uN = up[2:, 1:-1]
    uS = up[:-2, 1:-1]
    out = (aE + aW + aN + aS) * u - aE * uE - aW * uW - aN * uN - aS * uS
    return out / (h * h)


def dense_A(k: np.ndarray) -> np.ndarray:
    """The same matrix as ``apply_A``, assembled row by row as an explicit n x n array.

    Written independently of ``face_coefficients``: for every node P and each of its four
    neighbours Q the face coefficient is formed on the spot (harmonic mean if Q is
    interior, k_P if Q lies on the boundary), added to A_PP and, for interior Q,
    subtracted from A_PQ.
    """
    N = k.shape[0]
    n = N * N
    h = grid_h(N)
    A = np.zeros((n, n))
    for q in range(N):
        for p in range(N):
            row = q * N + p
            kp = k[q, p]
            for dp, dq in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                pp, qq = p + dp, q + dq
                if 0 <= pp < N and 0 <= qq < N:
                    kq = k[qq, pp]
                    a = 2.0 * kp * kq / (kp + kq)
                    A[row, row] += a
                    A[row, qq * N + pp] -= a
                else:
                    A[row, row] += kp
    return A / (h * h)


def energy_norm(k: np.ndarray, e: np.ndarray) -> float:
    """||e||_A = sqrt((e, A e)) (Theorem 1 notation)."""
    return math.sqrt(float(np.sum(e * apply_A(k, e))))


# ---------------------------------------------------------------------------------------
# Flexible conjugate gradients (Algorithm 1, Section 2.3)
# ---------------------------------------------------------------------------------------
def truncation_window(i: int, m_max: int) -> int:
    """m_i = min(i, max(1, i mod (m_max + 1))) of Algorithm 1."""
    return min(i, max(1, i % (m_max + 1)))


def _dot(a, b) -> float:
    return float(np.sum(a * b))


def fcg(A, B, f, u0, m_max: int, iters: int, tol: float | None = None, record: bool = False, dot=_dot):
    """Algorithm 1 (flexible CG) with preconditioner B, operator A (callables on arrays).

    Iteration i: w_i = B(r_i); m_i from the truncation rule; p_i = w_i minus the
    A-projections of w_i on the m_i previous directions (coefficients (w_i, s_k)/(p_k, s_k),
    all taken from w_i); s_i = A p_i; u and r updated with alpha = (p_i, r_i)/(p_i, s_i).
    Stops after ``iters`` iterations, or earlier when ||r_{i+1}|| <= tol ||r_0||.
    Returns a dict with u, r, iterations, relres history and (if record) every u_i, r_i,
    p_i, s_i. ``dot`` computes the inner products (default: numpy's pairwise sum); tests
    pass an exactly rounded one to measure how much the iterates depend on rounding.
    """
    u = np.array(u0, dtype=np.float64, copy=True)
    r = f - A(u)
    r0 = math.sqrt(dot(r, r))
    P, S, PS = [], [], []
    hist = [1.0 if r0 > 0 else 0.0]
    us, rs = [u.copy()], [r.copy()]
    status = STATUS_RUNNING
    it = 0
    if r0 == 0.0:
        status = STATUS_CONVERGED
    for i in range(iters if status == STATUS_RUNNING else 0):
        w = B(r)
        m_i = truncation_window(i, m_max)
        beta = [dot(w, S[kk]) / PS[kk] for kk in range(i - m_i, i)]
        p = w.copy()
        for j, kk in enumerate(range(i - m_i, i)):
            p = p - beta[j] * P[kk]
        s = A(p)
        ps = dot(p, s)
        pr = dot(p, r)
        if not (ps != 0.0 and math.isfinite(ps) and math.isfinite(pr)):
            status = STATUS_BREAKDOWN
            break
        alpha = pr / ps
        u = u + alpha * p
        r = r - alpha * s
        P.append(p)
        S.append(s)
        PS.append(ps)
        it = i + 1
        rn = math.sqrt(dot(r, r))
        hist.append(rn / r0)
        if record:
            us.append(u.copy())
            rs.append(r.copy())
        if rn == 0.0 or (tol is not None and rn <= tol * r0):
            status = STATUS_CONVERGED
            break
    if status == STATUS_RUNNING:
        status = STATUS_MAXITER
    out = {"u": u, "r": r, "iterations": it, "relres": np.array(hist), "status": status, "r0": r0}
    if record:
        out.update({"us": us, "rs": rs, "ps": P, "ss": S})
    return out


def cg_textbook(A, f, u0, iters: int, tol: float | None = None):
    """Hestenes-Stiefel conjugate gradients (the B = I reference of Fig. 2(a))."""
    u = np.array(u0, dtype=np.float64, copy=True)
    r = f - A(u)
    r0 = math.sqrt(float(np.sum(r * r)))
    d = r.copy()
    rr = float(np.sum(r * r))
    us = [u.copy()]
    it = 0
    for i in range(iters):
        Ad = A(d)
        alpha = rr / float(np.sum(d * Ad))
        u = u + alpha * d
        r = r - alpha * Ad
        rr_new = float(np.sum(r * r))
        d = r + (rr_new / rr) * d
        rr = rr_new
        us.append(u.copy())
        it = i + 1
        if tol is not None and math.sqrt(rr) <= tol * r0:
            break
    return {"u": u, "r": r, "iterations": it, "us": us}


def pcg_textbook(A, Minv, f, u0, iters: int):
    """Preconditioned CG with a fixed SPD linear preconditioner M^-1 (textbook form)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    r = f - A(u)
    z = Minv(r)
    d = z.copy()
    rz = float(np.sum(r * z))
    us = [u.copy()]
    for _ in range(iters):
        Ad = A(d)
        alpha = rz / float(np.sum(d * Ad))
        u = u + alpha * d
        r = r - alpha * Ad
        z = Minv(r)
        rz_new = float(np.sum(r * z))
        d = z + (rz_new / rz) * d
        rz = rz_new
        us.append(u.copy())
    return {"u": u, "us": us}


def jacobi_precond(k: np.ndarray, r: np.ndarray, steps: int) -> np.ndarray:
    """Jacobi(k) as a preconditioner, Eq. (15): x <- x + D(A)^-1 (r - A x), x^0 = 0."""
    N = k.shape[0]
    h = grid_h(N)
    aE, aW, aN, aS = face_coefficients(k)
    diag = (aE + aW + aN + aS) / (h * h)
    x = np.zeros_like(r)
    for _ in range(steps):
        x = x + (r - apply_A(k, x)) / diag
    return x


# ---------------------------------------------------------------------------------------
# Fourier neural operator (Section 2.4.2 and Appendix A)
# ---------------------------------------------------------------------------------------
def kx_frequencies(M: int) -> np.ndarray:
    """Signed x1-frequencies kept by the truncated transform: 0..M-1, then -M..-1."""
    return np.concatenate([np.arange(M), np.arange(-M, 0)])


def _twiddle(freqs: np.ndarray, N: int, sign: float) -> np.ndarray:
    """exp(sign * 2 pi i f x / N) for f in freqs (rows) and x = 0..N-1 (columns)."""
    x = np.arange(N)
    phase = np.mod(np.outer(freqs, x), N) / N  # exact integer reduction before scaling
    return np.exp(sign * 2j * np.pi * phase)


def analysis(v: np.ndarray, M: int) -> np.ndarray:
    """Truncated Fourier analysis (the operator A of the spectral layer, Section 2.4.2).

    v: [N][N][C] real on the grid x = (p, q). Returns c [2M][M][C] complex,
    c(k1, k2) = (1/n) sum_{p,q} v(p, q) exp(-2 pi i (k1 p + k2 q) / N).
    """
    N = v.shape[0]
    E1 = _twiddle(kx_frequencies(M), N, -1.0)        # [2M][N] over p
    E2 = _twiddle(np.arange(M), N, -1.0)              # [M][N]  over q
    t = np.tensordot(E2, v, axes=([1], [0]))          # sum over q -> [k2][p][C]
    c = np.tensordot(E1, t, axes=([1], [1]))          # sum over p -> [k1][k2][C]
    return c / (N * N)


def synthesis(c: np.ndarray, N: int) -> np.ndarray:
    """Truncated Fourier synthesis (the operator S, Section 2.4.2) for real fields.

    c: [2M][M][C] complex. Returns v [N][N][C],
    v(p, q) = Re sum_{k1, k2} w_k2 c(k1, k2) exp(+2 pi i (k1 p + k2 q) / N), w_0 = 1,
    w_{k2 > 0} = 2 (each kept k2 > 0 column stands for itself and its conjugate mirror).
    """
    M = c.shape[1]
    F1 = _twiddle(kx_frequencies(M), N, 1.0)          # [2M][N]
    F2 = _twiddle(np.arange(M), N, 1.0)               # [M][N]
    w = np.full(M, 2.0)
    w[0] = 1.0
    t = np.tensordot(F1, c, axes=([0], [0]))          # sum over k1 -> [p][k2][C]
    t = t * w[None, :, None]
    v = np.tensordot(F2, t, axes=([0], [1]))          # sum over k2 -> [q][p][C]
    return np.real(v)


def mode_mix(c: np.ndarray, R: np.ndarray) -> np.ndarray:
    """The linear map L of the spectral kernel S L A: per retained mode a complex C x C
    matrix, c'(k)_o = sum_i c(k)_i R(k)_{i,o}. c: [2M][M][C], R: [2M][M][C][C] complex."""
    return np.einsum("jki,jkio->jko", c, R, optimize=True)


def gelu(x: np.ndarray) -> np.ndarray:
    """GELU activation (Appendix A), exact form 0.5 x (1 + erf(x / sqrt 2))."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def unpack_weights(blob: np.ndarray, desc) -> dict:
    """Split the flat weight blob into float64 arrays (layout documented with ModelDesc)."""
    C, Cp, L, M, ci = desc.width, desc.proj_width, desc.layers, desc.modes, desc.in_channels
    b = np.asarray(blob, dtype=np.float64)
    pos = 0

    def take(shape):
        nonlocal pos
        size = int(np.prod(shape))
        out = b[pos:pos + size].reshape(shape)
        pos += size
        return out

    P = {"lift_w": take((C, ci)), "lift_b": take((C,)), "layers": []}
    for _ in range(L):
        W = take((C, C))
        bb = take((C,))
        R = take((2 * M, M, C, C, 2))
        P["layers"].append({"w": W, "b": bb, "r": R[..., 0] + 1j * R[..., 1]})
    P["proj1_w"] = take((Cp, C))
    P["proj1_b"] = take((Cp,))
    P["proj2_w"] = take((Cp,))
    P["proj2_b"] = take((1,))
    assert pos == b.size, (pos, b.size)
    return P


def fourier_layer(v: np.ndarray, layer: dict, M: int, activate: bool) -> np.ndarray:
    """One Fourier layer: act(W v + b + S L A v) with L = per-mode mixing by R."""
    N = v.shape[0]
    spec = synthesis(mode_mix(analysis(v, M), layer["r"]), N)
    h = (v @ layer["w"].T) + layer["b"] + spec
    return gelu(h) if activate else h


def no_forward(params: dict, desc, r: np.ndarray, logk: np.ndarray) -> np.ndarray:
    """The preconditioner z = NO(r, log k) of Algorithm 1 (w_i = B(r_i)), Appendix A.

    r, logk: [N][N]. Encoder: v0 = lift_w [r/rms, log k] + lift_b. Processor: the Fourier
    layers, GELU after all but the last. Decoder: proj2_w . GELU(proj1_w v + proj1_b) +
    proj2_b. Output multiplied by output_scale(...); zero when r = 0.
    """
    rms = math.sqrt(float(np.mean(r * r)))
    if rms == 0.0:
        return np.zeros_like(r)
    x = np.stack([r / rms, logk], axis=-1)
    v = x @ params["lift_w"].T + params["lift_b"]
    L = len(params["layers"])
    for l, layer in enumerate(params["layers"]):
        v = fourier_layer(v, layer, desc.modes, activate=(l < L - 1))
    hid = gelu(v @ params["proj1_w"].T + params["proj1_b"])
    zt = hid @ params["proj2_w"] + params["proj2_b"][0]
    return output_scale(desc, rms, logk) * zt


def output_scale(desc, rms: float, logk: np.ndarray):
    """Factor that puts the decoder output into the units of A^-1: h^2 rms(r), divided by k at
    every grid point when desc.output_scale is 1 (a scalar, or an [N][N] array)."""
    base = grid_h(logk.shape[0]) ** 2 * rms
    return base * np.exp(-logk) if getattr(desc, "output_scale", 0) else base


# ---------------------------------------------------------------------------------------
# Losses (Section 3.1, Eq. (11)-(12))
# ---------------------------------------------------------------------------------------
def notay_loss(ks, zs, es) -> float:
    """Eq. (11): mean over samples of ||z - e||_A / ||e||_A (A from each sample's k)."""
    vals = [energy_norm(k, z - e) / energy_norm(k, e) for k, z, e in zip(ks, zs, es)]
    return float(np.mean(vals))


def l2_loss(zs, es) -> float:
    """Eq. (12): mean over samples of ||z - e||_2 / ||e||_2."""
    vals = [np.linalg.norm(z - e) / np.linalg.norm(e) for z, e in zip(zs, es)]
    return float(np.mean(vals))


# ---------------------------------------------------------------------------------------
# Training gradient of the energy-norm loss (Eq. (11)), hand-written reverse mode
# ---------------------------------------------------------------------------------------
def synthesis_adjoint(g: np.ndarray, M: int) -> np.ndarray:
    """Adjoint of ``synthesis`` w.r.t. its complex input read as (re, im) pairs:
    dc(k) = w_k2 sum_x g(x) exp(-2 pi i k.x / N), g: [N][N][C] -> [2M][M][C]."""
    N = g.shape[0]
    E1 = _twiddle(kx_frequencies(M), N, -1.0)
    E2 = _twiddle(np.arange(M), N, -1.0)
    w = np.full(M, 2.0)
    w[0] = 1.0
    t = np.tensordot(E2, g, axes=([1], [0]))
    c = np.tensordot(E1, t, axes=([1], [1]))
    return c * w[None, :, None]


def analysis_adjoint(dc: np.ndarray, N: int) -> np.ndarray:
    """Adjoint of ``analysis`` (real input) w.r.t. its (re, im) outputs:
    dv(x) = (1/n) sum_k Re(dc(k) exp(+2 pi i k.x / N)), dc: [2M][M][C] -> [N][N][C]."""
    M = dc.shape[1]
    F1 = _twiddle(kx_frequencies(M), N, 1.0)
    F2 = _twiddle(np.arange(M), N, 1.0)
    t = np.tensordot(F1, dc, axes=([0], [0]))
    v = np.tensordot(F2, t, axes=([0], [1]))
    return np.real(v) / (N * N)


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d/dx GELU(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _forward_saved(params: dict, desc, r: np.ndarray, logk: np.ndarray) -> dict:
    rms = math.sqrt(float(np.mean(r * r)))
    x0 = np.stack([r / rms, logk], axis=-1)
    v = x0 @ params["lift_w"].T + params["lift_b"]
    vs, hs, cs = [v], [], []
    L = len(params["layers"])
    for l, layer in enumerate(params["layers"]):
        c = analysis(v, desc.modes)
        h = v @ layer["w"].T + layer["b"] + synthesis(mode_mix(c, layer["r"]), v.shape[0])
        v = gelu(h) if l < L - 1 else h
        cs.append(c)
        hs.append(h)
        vs.append(v)
    a = v @ params["proj1_w"].T + params["proj1_b"]
    g = gelu(a)
    zt = g @ params["proj2_w"] + params["proj2_b"][0]
    scale = output_scale(desc, rms, logk)
    return {"rms": rms, "scale": scale, "x0": x0, "vs": vs, "hs": hs, "cs": cs, "a": a, "g": g, "z": scale * zt}


def notay_loss_and_grad(params: dict, desc, ks, rs, es):
    """Eq. (11) over a batch: L = mean_j ||z_j - e_j||_A / ||e_j||_A with z_j = NO(r_j, log k_j),
    and dL/d(weights) as a flat float64 array in the weight-blob order.

    dL/dz_j = A (z_j - e_j) / (||z_j - e_j||_A ||e_j||_A) / batch; the rest is the chain rule
    through the decoder, the Fourier layers (pointwise path, the per-mode mixing and the
    adjoints of the truncated transforms) and the encoder.
    """
    return _loss_and_grad(params, desc, ks, rs, es, energy=True)


def l2_loss_and_grad(params: dict, desc, ks, rs, es):
    """The L2 loss in error form (the ablation loss of Section 3.1, compared with Eq. (11) in
    Section 3.4): L = mean_j ||z_j - e_j||_2 / ||e_j||_2, and its gradient in blob order.
    dL/dz_j = (z_j - e_j) / (||z_j - e_j||_2 ||e_j||_2) / batch; the chain rule below dz is the
    same as for Eq. (11)."""
    return _loss_and_grad(params, desc, ks, rs, es, energy=False)


def _loss_and_grad(params: dict, desc, ks, rs, es, energy: bool):
    """Shared reverse mode of the two losses: the norm is the A-norm (energy) or the 2-norm."""
    L = len(params["layers"])
    grads = {k: np.zeros_like(params[k]) for k in ("lift_w", "lift_b", "proj1_w", "proj1_b", "proj2_w", "proj2_b")}
    glayers = [{"w": np.zeros_like(p["w"]), "b": np.zeros_like(p["b"]), "r": np.zeros_like(p["r"])}
               for p in params["layers"]]
    B = len(ks)
    loss = 0.0
    for k, r, e in zip(ks, rs, es):
        S = _forward_saved(params, desc, r, np.log(k))
        d = S["z"] - e
        Ad = apply_A(k, d) if energy else d
        nd = math.sqrt(float(np.sum(d * Ad)))
        ne = energy_norm(k, e) if energy else float(np.linalg.norm(e))
        loss += nd / ne / B
        dz = Ad / (nd * ne) / B
        dzt = S["scale"] * dz
        grads["proj2_w"] += np.einsum("qp,qph->h", dzt, S["g"])
        grads["proj2_b"] += np.sum(dzt)
        da = dzt[..., None] * params["proj2_w"] * gelu_grad(S["a"])
        grads["proj1_w"] += np.einsum("qph,qpc->hc", da, S["vs"][L])
        grads["proj1_b"] += np.sum(da, axis=(0, 1))
        dv = da @ params["proj1_w"]
        for l in range(L - 1, -1, -1):
            layer = params["layers"][l]
            dh = dv * gelu_grad(S["hs"][l]) if l < L - 1 else dv
            glayers[l]["w"] += np.einsum("qpo,qpi->oi", dh, S["vs"][l])
            glayers[l]["b"] += np.sum(dh, axis=(0, 1))
            dcp = synthesis_adjoint(dh, desc.modes)                              # d/d c'
            glayers[l]["r"] += np.einsum("jki,jko->jkio", np.conj(S["cs"][l]), dcp)
            dc = np.einsum("jkio,jko->jki", np.conj(layer["r"]), dcp)             # d/d c
            dv = dh @ layer["w"] + analysis_adjoint(dc, r.shape[0])
        grads["lift_w"] += np.einsum("qpc,qpi->ci", dv, S["x0"])
        grads["lift_b"] += np.sum(dv, axis=(0, 1))
    parts = [grads["lift_w"].ravel(), grads["lift_b"].ravel()]
    for gl in glayers:
        parts += [gl["w"].ravel(), gl["b"].ravel(), np.stack([gl["r"].real, gl["r"].imag], axis=-1).ravel()]
    parts += [grads["proj1_w"].ravel(), grads["proj1_b"].ravel(), grads["proj2_w"].ravel(), grads["proj2_b"].ravel()]
    return loss, np.concatenate(parts)
