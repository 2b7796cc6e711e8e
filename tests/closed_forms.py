"""Closed forms used by the pins of the discretisation (Eq. (1)-(2)), shared by the CPU pins
of the oracle and the GPU parity tests. Nothing here calls the oracle or the library."""
import math

import numpy as np


def layered_flux_field(N, axis=1, j=2, c=1.3, seed=0, contrast=3.0):
    """A coefficient layered along one axis and a grid function on which the five-point
    operator has a closed form at every node, fixed by flux balance alone.

    k depends only on the index along `axis` (axis=1: p, the x1 index; axis=0: q), with a
    log-uniform value per layer over a factor exp(2*contrast). Along that axis phi carries a
    constant flux c through every face: the two half cells between neighbouring nodes are
    resistances h/(2 k) in series, so phi rises by c * (h/(2 k_a) + h/(2 k_b)) from node a to
    node b, and the boundary face (node at distance h from the wall, coefficient k of the
    node) takes phi_0 = c h / k_0. Across the other axis u is the discrete sine mode
    psi = sin(j pi h (t + 1)), which vanishes on both walls.

    For u = phi (x) psi the operator h^-2 sum_faces a_f (u_P - u_Q) then gives
      (A u) = h^-2 psi [ 2 (1 - cos(j pi h)) k phi ]                  at all but the last layer,
      (A u) = h^-2 psi [ 2 (1 - cos(j pi h)) k phi + k phi + c h ]    at the last layer,
    because the flux entering each node along `axis` equals the flux leaving it. That holds
    only if every interior face coefficient is 1 / (mean of 1/k) over its two half cells
    (the harmonic mean) and a boundary face takes k of its node. Returns (k, u, A u), each
    [N][N] indexed [q][p].
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (N + 1)
    kl = np.exp(rng.uniform(-contrast, contrast, N))
    phi = np.empty(N)
    phi[0] = c * h / kl[0]
    for t in range(N - 1):
        phi[t + 1] = phi[t] + c * (0.5 * h / kl[t] + 0.5 * h / kl[t + 1])
    psi = np.array([math.sin(j * math.pi * h * (t + 1)) for t in range(N)])
    lam = 2.0 * (1.0 - math.cos(j * math.pi * h))
    ew = lam * kl * phi                      # along-axis balance leaves only the cross term
    ew[N - 1] += kl[N - 1] * phi[N - 1] + c * h
    if axis == 1:
        k = np.tile(kl, (N, 1))
        u = np.outer(psi, phi)
        Au = np.outer(psi, ew) / (h * h)
    else:
        k = np.tile(kl[:, None], (1, N))
        u = np.outer(phi, psi)
        Au = np.outer(ew, psi) / (h * h)
    return k, u, Au
