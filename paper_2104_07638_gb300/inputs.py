"""Seeded synthetic inputs for the all-principal-minor path.

This module only draws random numbers and evaluates free-particle Green's
functions (the matrix *entries*); it contains none of the minor, connected-sum,
Keldysh-sum or permanent arithmetic. Both the CUDA path and the CPU oracle take
their inputs from here, so that the two see bit-identical matrices.

Workloads (matrix entries are Green's functions G0(X_i - X_j) of vertices X_i,
as in the CDet weight of Section V.A and the Keldysh block matrix of Section V.D):

* ``gaussian_plus_2I``   -- A_ij ~ N(0,1) + 2 delta_ij (dense, well conditioned).
* ``hubbard_batch``      -- free 2D square-lattice Hubbard G0 (t=1, mu=-0.5, beta=5,
                            32x32 k-grid), vertices r uniform in an 8x8 window and
                            tau uniform on a 2^14-point grid of [0, beta).
* ``keldysh_batch``      -- 2n x 2n complex block matrices of a free 1D chain
                            (eps_k=-2cos k, mu=0, beta=10, 256 k-points), sites
                            uniform in {0..7}, real times on a 2^14-point grid of [0,4].
* ``perm_batch``         -- A_ij ~ U(0,1) times a symmetric 0/1 mask with 30% zeros
                            off the diagonal.
* ``varlen_orders``      -- orders n uniform in {4..16} for uneven batches.

Times are drawn on a fine grid (distinct within one matrix) so that every time
difference is an exact grid multiple and G0 can be read from a table computed
once by the k-sum; ties (and with them the equal-time ambiguity) never occur off
the diagonal.
"""
from __future__ import annotations

import functools

import numpy as np

# ----------------------------------------------------------------------------
# generic
# ----------------------------------------------------------------------------


def gaussian_plus_2I(n: int, batch: int = 1, seed: int = 1) -> np.ndarray:
    """A_ij ~ N(0,1) + 2*delta_ij, shape (batch, n, n), float64."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, n, n))
    A += 2.0 * np.eye(n)[None]
    return A


def perm_batch(n: int = 14, batch: int = 4096, seed: int = 4,
               p_zero: float = 0.3) -> np.ndarray:
    """A_ij ~ U(0,1) times a symmetric mask: each unordered pair i<j is zeroed
    (both (i,j) and (j,i)) with probability p_zero; the diagonal is kept."""
    rng = np.random.default_rng(seed)
    A = rng.random((batch, n, n))
    keep = rng.random((batch, n, n)) >= p_zero
    iu = np.triu_indices(n, 1)
    m = np.ones((batch, n, n), dtype=bool)
    m[:, iu[0], iu[1]] = keep[:, iu[0], iu[1]]
    m[:, iu[1], iu[0]] = keep[:, iu[0], iu[1]]
    return A * m


def varlen_orders(batch: int, lo: int = 4, hi: int = 16, seed: int = 3) -> np.ndarray:
    """Orders n uniform in {lo..hi}, int32."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=batch).astype(np.int32)


def _distinct_grid_indices(rng, batch: int, n: int, M: int) -> np.ndarray:
    """batch x n integer grid indices in [0, M), distinct within each row."""
    idx = rng.integers(0, M, size=(batch, n))
    while True:
        s = np.sort(idx, axis=1)
        bad = np.any(s[:, 1:] == s[:, :-1], axis=1) if n > 1 else np.zeros(batch, bool)
        if not bad.any():
            return idx
        idx[bad] = rng.integers(0, M, size=(int(bad.sum()), n))


# ----------------------------------------------------------------------------
# 2D Hubbard G0 (imaginary time)
# ----------------------------------------------------------------------------

HUB_T, HUB_MU, HUB_BETA, HUB_NK, HUB_WIN = 1.0, -0.5, 5.0, 32, 8
HUB_MTAU = 1 << 14


@functools.lru_cache(maxsize=None)
def hubbard_g0_table(t: float = HUB_T, mu: float = HUB_MU, beta: float = HUB_BETA,
                     nk: int = HUB_NK, win: int = HUB_WIN, mtau: int = HUB_MTAU):
    """G0(r, tau) of the free 2D square-lattice Hubbard model for |rx|,|ry| < win
    and tau = d*beta/mtau, d in [-(mtau-1), mtau-1].

    Convention G(r,tau) = -<T c_r(tau) c_0^+(0)>, xi_k = -2t(cos kx + cos ky) - mu:
      0 < tau < beta :  G0 = -(1/N) sum_k cos(k.r) e^{-xi tau} (1 - f(xi))
     -beta < tau < 0 :  G0 = +(1/N) sum_k cos(k.r) e^{-xi tau} f(xi)
      tau = 0        :  the 0^- limit, G0(0,0^-) = density n_sigma.
    Returns an array of shape (win, win, 2*mtau-1); index [|rx|, |ry|, d+mtau-1].
    Both exponentials are evaluated in overflow-free form.
    """
    m = np.arange(nk)
    # kx classes m and nk-m share cos; weight 2 unless m in {0, nk/2}
    half = np.arange(nk // 2 + 1)
    w1 = np.where((half == 0) | (half == nk // 2), 1.0, 2.0)
    k1 = 2.0 * np.pi * half / nk
    kx, ky = np.meshgrid(k1, k1, indexing="ij")
    wk = np.outer(w1, w1).ravel()
    xi = (-2.0 * t * (np.cos(kx) + np.cos(ky)) - mu).ravel()
    r = np.arange(win)
    cosx = np.cos(np.outer(r, k1))                                     # (win, nkh)
    W = (cosx[:, None, :, None] * cosx[None, :, None, :]).reshape(win * win, -1)
    W = W * wk[None, :] / float(nk * nk)                                # (win^2, K)
    d = np.arange(-(mtau - 1), mtau)
    tau = d * (beta / mtau)
    pos = tau > 0
    tp = tau[pos][None, :]
    xi_c = xi[:, None]
    # e^{-xi tau} (1-f) = e^{-xi tau}/(1+e^{-beta xi}); for xi<0 rewrite as e^{xi(beta-tau)}/(1+e^{beta xi})
    Ep = np.where(xi_c >= 0,
                  np.exp(-xi_c * tp) / (1.0 + np.exp(-beta * np.abs(xi_c))),
                  np.exp(xi_c * (beta - tp)) / (1.0 + np.exp(-beta * np.abs(xi_c))))
    tn = -tau[~pos][None, :]                                            # s = -tau in [0, beta)
    # e^{xi s} f = e^{xi s}/(e^{beta xi}+1); for xi>0 rewrite as e^{xi(s-beta)}/(1+e^{-beta xi})
    En = np.where(xi_c <= 0,
                  np.exp(xi_c * tn) / (1.0 + np.exp(-beta * np.abs(xi_c))),
                  np.exp(xi_c * (tn - beta)) / (1.0 + np.exp(-beta * np.abs(xi_c))))
    G = np.empty((win * win, d.size))
    G[:, pos] = -(W @ Ep)
    G[:, ~pos] = +(W @ En)
    return G.reshape(win, win, d.size)


def hubbard_vertices(batch: int, n: int, seed: int = 2, win: int = HUB_WIN,
                     mtau: int = HUB_MTAU):
    """Vertices (x, y, tau-grid-index), each (batch, n) int64; tau indices distinct."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, win, size=(batch, n))
    y = rng.integers(0, win, size=(batch, n))
    m = _distinct_grid_indices(rng, batch, n, mtau)
    return x, y, m


def hubbard_matrices_from_vertices(x, y, m, mtau: int = HUB_MTAU) -> np.ndarray:
    """(M)_ij = G0(r_i - r_j, tau_i - tau_j); diagonal = G0(0, 0^-)."""
    G = hubbard_g0_table(mtau=mtau)
    dx = np.abs(x[:, :, None] - x[:, None, :])
    dy = np.abs(y[:, :, None] - y[:, None, :])
    dt = m[:, :, None] - m[:, None, :] + (mtau - 1)
    return G[dx, dy, dt]


def hubbard_batch(batch: int = 65536, n: int = 12, seed: int = 2) -> np.ndarray:
    """Hubbard G0 matrices, shape (batch, n, n), float64."""
    x, y, m = hubbard_vertices(batch, n, seed)
    return hubbard_matrices_from_vertices(x, y, m)


def hubbard_batch_slice(total: int, n: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Matrices lo .. hi-1 of the seeded batch hubbard_batch(total, n, seed): the
    vertices of the whole batch are drawn (a few numbers per matrix), the
    matrices only for the slice, so that ranks holding contiguous slices hold
    exactly the one batch between them."""
    x, y, m = hubbard_vertices(total, n, seed)
    return hubbard_matrices_from_vertices(x[lo:hi], y[lo:hi], m[lo:hi])


def hubbard_varlen(orders: np.ndarray, seed: int = 3):
    """Packed Hubbard matrices of mixed order: returns (flat float64 array,
    int64 element offsets of each matrix)."""
    orders = np.asarray(orders, dtype=np.int64)
    off = np.zeros(orders.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(orders * orders)
    flat = np.empty(int(off[-1]))
    rng = np.random.default_rng(seed)
    for n in np.unique(orders):
        sel = np.nonzero(orders == n)[0]
        sub_seed = int(rng.integers(0, 2**63 - 1))
        A = hubbard_batch(sel.size, int(n), seed=sub_seed)
        for k, b in enumerate(sel):
            flat[off[b]:off[b + 1]] = A[k].ravel()
    return flat, off[:-1].copy()


# ----------------------------------------------------------------------------
# 1D chain Keldysh G0 (real time)
# ----------------------------------------------------------------------------

KEL_BETA, KEL_L, KEL_WIN, KEL_TMAX = 10.0, 256, 8, 4.0
KEL_MT = 1 << 14


@functools.lru_cache(maxsize=None)
def keldysh_g0_tables(beta: float = KEL_BETA, L: int = KEL_L, win: int = KEL_WIN,
                      tmax: float = KEL_TMAX, mt: int = KEL_MT, shift: float = 0.0):
    """G^<(x,t) and G^>(x,t) of a free 1D chain (eps_k = -2 cos k + shift, mu = 0;
    shift = +-h is a Zeeman field for the two spins):
        G^<(x,t) = +(i/L) sum_k e^{i(kx - eps_k t)} f(eps_k)
        G^>(x,t) = -(i/L) sum_k e^{i(kx - eps_k t)} (1 - f(eps_k))
    for |x| < win and t = d*tmax/mt, d in [-(mt-1), mt-1]. Returns two complex
    arrays of shape (win, 2*mt-1) indexed [|x|, d+mt-1] (G depends on |x| only)."""
    half = np.arange(L // 2 + 1)
    wk = np.where((half == 0) | (half == L // 2), 1.0, 2.0)
    k = 2.0 * np.pi * half / L
    eps = -2.0 * np.cos(k) + shift
    f = 1.0 / (np.exp(beta * eps) + 1.0)
    x = np.arange(win)
    C = np.cos(np.outer(x, k)) * wk[None, :] / float(L)               # (win, K)
    d = np.arange(-(mt - 1), mt)
    tt = d * (tmax / mt)
    ph = np.exp(-1j * np.outer(eps, tt))                                # (K, T)
    Gl = 1j * (C @ (ph * f[:, None]))
    Gg = -1j * (C @ (ph * (1.0 - f)[:, None]))
    return Gl, Gg


def keldysh_vertices(batch: int, n: int, seed: int = 3, win: int = KEL_WIN,
                     mt: int = KEL_MT):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, win, size=(batch, n))
    m = _distinct_grid_indices(rng, batch, n, mt)
    return x, m


def keldysh_matrices_from_vertices(x, m, mt: int = KEL_MT, shift: float = 0.0) -> np.ndarray:
    """2n x 2n complex block matrices; block (i,j) sits at rows 2i,2i+1 (Keldysh
    index +,-) and columns 2j,2j+1:
        [[G^{++}, G^{+-}], [G^{-+}, G^{--}]](x_i - x_j, t_i - t_j),
    G^{++}(t) = theta(t) G^>(t) + theta(-t) G^<(t), G^{--}(t) = theta(t) G^<(t) + theta(-t) G^>(t),
    G^{+-} = G^<, G^{-+} = G^>; at equal times (the diagonal blocks) G^{++} = G^{--} = G^<."""
    Gl, Gg = keldysh_g0_tables(mt=mt, shift=shift)
    batch, n = x.shape
    dx = np.abs(x[:, :, None] - x[:, None, :])
    dm = m[:, :, None] - m[:, None, :]
    gl = Gl[dx, dm + (mt - 1)]
    gg = Gg[dx, dm + (mt - 1)]
    later = dm > 0
    gpp = np.where(later, gg, gl)
    gmm = np.where(later, gl, gg)
    eye = np.eye(n, dtype=bool)[None]
    gmm = np.where(eye, gl, gmm)
    M = np.empty((batch, 2 * n, 2 * n), dtype=np.complex128)
    M[:, 0::2, 0::2] = gpp
    M[:, 0::2, 1::2] = gl
    M[:, 1::2, 0::2] = gg
    M[:, 1::2, 1::2] = gmm
    return M


def keldysh_batch(batch: int, n: int, seed: int = 3) -> np.ndarray:
    x, m = keldysh_vertices(batch, n, seed)
    return keldysh_matrices_from_vertices(x, m)


def keldysh_varlen(orders: np.ndarray, seed: int = 3):
    """Packed Keldysh block matrices of mixed order: (flat complex128 array,
    int64 element offsets in complex units)."""
    orders = np.asarray(orders, dtype=np.int64)
    off = np.zeros(orders.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(4 * orders * orders)
    flat = np.empty(int(off[-1]), dtype=np.complex128)
    rng = np.random.default_rng(seed)
    for n in np.unique(orders):
        sel = np.nonzero(orders == n)[0]
        sub_seed = int(rng.integers(0, 2**63 - 1))
        M = keldysh_batch(sel.size, int(n), seed=sub_seed)
        for k, b in enumerate(sel):
            flat[off[b]:off[b + 1]] = M[k].ravel()
    return flat, off[:-1].copy()


# --- Nambu (BCS) matrices for the XNOR minors / Nambu CDet -------------------
NAMBU_DELTA = 0.3
NAMBU_MTAU = 1 << 12


def nambu_g0_table(t: float = HUB_T, mu: float = HUB_MU, beta: float = HUB_BETA, delta: float = NAMBU_DELTA,
                   nk: int = HUB_NK, win: int = HUB_WIN, mtau: int = NAMBU_MTAU):
    """Bare Nambu propagator of the 2D square-lattice attractive Hubbard model at
    the BCS mean field, for |rx|,|ry| < win and tau = d*beta/mtau.

    Nambu spinor psi_k = (c_k,up, c^+_-k,down), h_k = [[xi, delta], [delta, -xi]],
    E = sqrt(xi^2 + delta^2), projectors P+- = (1 +- h/E)/2. With
    G(k,tau) = -<T psi_k(tau) psi_k^+(0)>:
      0 < tau < beta : G = -(P+ e^{-E tau} + P- e^{-E(beta-tau)}) / (1 + e^{-beta E})
     -beta < tau < 0 : G(k,tau) = -G(k,tau+beta)
      tau = 0        : the 0^- limit, G = n_F(h_k).
    Real space: G(r,tau) = (1/N) sum_k cos(k.r) G(k,tau) (real). Every
    exponential has a non-positive argument. Returns (win, win, 2*mtau-1, 2, 2).
    """
    half = np.arange(nk // 2 + 1)
    w1 = np.where((half == 0) | (half == nk // 2), 1.0, 2.0)
    k1 = 2.0 * np.pi * half / nk
    kx, ky = np.meshgrid(k1, k1, indexing="ij")
    wk = np.outer(w1, w1).ravel()
    xi = (-2.0 * t * (np.cos(kx) + np.cos(ky)) - mu).ravel()
    E = np.sqrt(xi * xi + delta * delta)
    r = np.arange(win)
    cosx = np.cos(np.outer(r, k1))
    W = (cosx[:, None, :, None] * cosx[None, :, None, :]).reshape(win * win, -1)
    W = W * wk[None, :] / float(nk * nk)                                # (win^2, K)
    d = np.arange(-(mtau - 1), mtau)
    tau = d * (beta / mtau)
    # s in (0, beta]: tau > 0 -> s = tau with sign -1; tau <= 0 -> s = tau + beta with sign +1
    # (tau = 0 is the 0^- limit: s = beta)
    s = np.where(tau > 0, tau, tau + beta)[None, :]
    sgn = np.where(tau > 0, -1.0, 1.0)[None, :]
    Ec = E[:, None]
    den = 1.0 + np.exp(-beta * Ec)
    ep = np.exp(-Ec * s) / den                  # weight of P+
    em = np.exp(-Ec * (beta - s)) / den         # weight of P-
    u2 = (0.5 * (1.0 + xi / E))[:, None]
    v2 = (0.5 * (1.0 - xi / E))[:, None]
    g = (0.5 * delta / E)[:, None]
    G = np.empty((win * win, d.size, 2, 2))
    G[:, :, 0, 0] = sgn * (W @ (u2 * ep + v2 * em))
    G[:, :, 1, 1] = sgn * (W @ (v2 * ep + u2 * em))
    G[:, :, 0, 1] = sgn * (W @ (g * (ep - em)))
    G[:, :, 1, 0] = G[:, :, 0, 1]
    return G.reshape(win, win, d.size, 2, 2)


def nambu_matrices_from_vertices(x, y, m, mtau: int = NAMBU_MTAU) -> np.ndarray:
    """2n x 2n matrices of 2 x 2 blocks: block (i, j) at rows 2i, 2i+1 and
    columns 2j, 2j+1 is G(r_i - r_j, tau_i - tau_j); diagonal blocks G(0, 0^-)."""
    G = nambu_g0_table(mtau=mtau)
    b, n = x.shape
    dx = np.abs(x[:, :, None] - x[:, None, :])
    dy = np.abs(y[:, :, None] - y[:, None, :])
    dt = m[:, :, None] - m[:, None, :] + (mtau - 1)
    blocks = G[dx, dy, dt]                                              # (b, n, n, 2, 2)
    return np.ascontiguousarray(blocks.transpose(0, 1, 3, 2, 4).reshape(b, 2 * n, 2 * n))


def nambu_batch(batch: int = 65536, n: int = 12, seed: int = 6) -> np.ndarray:
    """Nambu G0 matrices, shape (batch, 2n, 2n), float64 (vertices as for the
    Hubbard batches: sites on the 8 x 8 window, distinct times on the grid)."""
    x, y, m = hubbard_vertices(batch, n, seed, mtau=NAMBU_MTAU)
    return nambu_matrices_from_vertices(x, y, m)


# --- two vertex types (NAND minors, Section III.C / V.C) -----------------------

def two_type_batch(batch: int = 4096, n: int = 10, seed: int = 7) -> np.ndarray:
    """Hubbard G0 matrices for expansions with two vertex types, shape
    (batch, 2n, 2n): vertex i at (r_i, tau_i) (as hubbard_batch) has its second
    type at (r_i + e_x, tau_i), a translated copy (the artificial second vertex
    of Section V.C); row/column 2i is type 1, 2i+1 type 2, entry
    G0(X_i^a - X_j^b), equal-time entries G0(r, 0^-)."""
    x, y, m = hubbard_vertices(batch, n, seed)
    G = hubbard_g0_table(win=HUB_WIN + 1)
    xs = np.stack([x, x + 1], axis=-1).reshape(batch, 2 * n)
    ys = np.repeat(y, 2, axis=-1)
    ms = np.repeat(m, 2, axis=-1)
    dx = np.abs(xs[:, :, None] - xs[:, None, :])
    dy = np.abs(ys[:, :, None] - ys[:, None, :])
    dt = ms[:, :, None] - ms[:, None, :] + (HUB_MTAU - 1)
    return np.ascontiguousarray(G[dx, dy, dt])


# --- two spins under one Keldysh assignment (Section V.D with Eq. CTINT) -------
KEL_ZEEMAN = 0.5


def keldysh2_batch(batch: int, n: int, seed: int = 8, h: float = KEL_ZEEMAN):
    """Two Keldysh block matrices per vertex set, (up, down), each (batch, 2n, 2n)
    complex128: the chain of keldysh_batch with the energies shifted by -h (up)
    and +h (down), the same vertices for both spins."""
    x, m = keldysh_vertices(batch, n, seed)
    return keldysh_matrices_from_vertices(x, m, shift=-h), keldysh_matrices_from_vertices(x, m, shift=h)
