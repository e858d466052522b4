"""Seeded synthetic inputs for the THC second-order-exchange workloads.

This module builds INPUTS only: a Hamiltonian, its imaginary-time Green's
function G(tau) on a Chebyshev-Lobatto grid, a THC collocation matrix X and a
positive semidefinite THC metric V.  It holds none of the self-energy
arithmetic; both the CPU oracle and the CUDA path consume what it returns.

Shapes follow the library's layout (row-major, outermost first):

* ``G``   ``[n_spin][n_k][n_tau][n][n]``  (float64 for molecules, complex128 for solids)
* ``X``   ``[n_k][N][n]``  with ``X[k][P][p]`` = X^k_{pP} of the THC factorisation (Sec. II C)
* ``V``   ``[n_q][N][N]``  the THC metric U^q_{PQ} (Sec. II C), one block per momentum transfer
* ``tau`` ``[n_tau]``  Chebyshev-Lobatto nodes on [0, beta], symmetric under tau -> beta - tau

Generator recipe (the paper's molecules/solids are replaced by these stand-ins):

* H0: A ~ N(0,1)^{n x n}, H = (A + A^T)/2, eigenvalues mapped affinely to [-2, 2] Ha,
  eigenvectors kept.  mu sits midway between eigenvalues n/2 and n/2+1 (1-based).
* G(tau) = -U diag(e^{-xi tau} / (1 + e^{-beta xi})) U^T with xi = eps - mu, evaluated in
  the overflow-safe form for xi <= 0.
* X[P, p] ~ N(0,1)/sqrt(n).
* V = Z Z^T with Z ~ N(0,1)^{N x N}, column k rescaled to norm 1/(1+k).
* Seeds: ``numpy.random.default_rng(2412188290 + 10*c + stream)``, streams 0=H0, 1=X, 2=Z,
  3=spin/k extras, 4=batch sizes; instance i of a batch uses the seed list [that, i].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2412188290


def _rng(cfg: int, stream: int, instance: int | None = None) -> np.random.Generator:
    s = SEED_BASE + 10 * cfg + stream
    return np.random.default_rng([s, instance] if instance is not None else s)


def tau_nodes(n_tau: int, beta: float) -> np.ndarray:
    """Chebyshev-Lobatto nodes tau_j = (beta/2)(1 - cos(pi j/(n_tau-1))) on [0, beta]."""
    if n_tau < 2:
        raise ValueError("n_tau must be >= 2")
    j = np.arange(n_tau)
    t = 0.5 * beta * (1.0 - np.cos(np.pi * j / (n_tau - 1)))
    t[0], t[-1] = 0.0, beta
    # exact mirror symmetry tau_{n-1-j} = beta - tau_j
    half = n_tau // 2
    t[n_tau - 1 - np.arange(half)] = beta - t[np.arange(half)]
    if n_tau % 2:
        t[half] = 0.5 * beta
    return t


def random_hamiltonian(rng: np.random.Generator, n: int, lo: float = -2.0, hi: float = 2.0):
    """Real symmetric n x n matrix with spectrum mapped affinely onto [lo, hi]."""
    a = rng.standard_normal((n, n))
    h = 0.5 * (a + a.T)
    e, u = np.linalg.eigh(h)
    if n == 1:
        e2 = np.array([0.5 * (lo + hi)])
    else:
        e2 = lo + (e - e[0]) * (hi - lo) / (e[-1] - e[0])
    return (u * e2) @ u.T, e2, u


def half_filling_mu(eps_sorted: np.ndarray) -> float:
    n = eps_sorted.size
    if n == 1:
        return float(eps_sorted[0]) + 1.0
    m = n // 2
    return 0.5 * (eps_sorted[m - 1] + eps_sorted[m])


def fermi_propagator_diag(xi: np.ndarray, tau: np.ndarray, beta: float) -> np.ndarray:
    """f[j, i] = e^{-xi_i tau_j} / (1 + e^{-beta xi_i}), overflow safe for either sign of xi."""
    xi = np.asarray(xi, dtype=np.float64)[None, :]
    t = np.asarray(tau, dtype=np.float64)[:, None]
    pos = xi > 0
    with np.errstate(over="ignore", under="ignore"):
        fp = np.exp(-np.where(pos, xi, 0.0) * t) / (1.0 + np.exp(-beta * np.where(pos, xi, 0.0)))
        fn = np.exp(np.where(pos, 0.0, xi) * (beta - t)) / (1.0 + np.exp(beta * np.where(pos, 0.0, xi)))
    return np.where(pos, fp, fn)


def green_tau(eps: np.ndarray, u: np.ndarray, mu: float, tau: np.ndarray, beta: float) -> np.ndarray:
    """G(tau_j) = -U diag(f_j) U^H for every node; returns [n_tau][n][n]."""
    f = fermi_propagator_diag(eps - mu, tau, beta)
    return -np.einsum("pi,ji,qi->jpq", u, f, u.conj(), optimize=True)


def decaying_metric(rng: np.random.Generator, N: int, complex_: bool = False) -> np.ndarray:
    """Z with columns of norm 1/(1+k); returns Z (the metric is Z Z^H)."""
    if complex_:
        z = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(2.0)
    else:
        z = rng.standard_normal((N, N))
    norms = np.linalg.norm(z, axis=0)
    z = z / norms[None, :] / (1.0 + np.arange(N))[None, :]
    return z


@dataclass
class Workload:
    """One problem instance in the library's layout (see module docstring)."""

    name: str
    n: int
    N: int
    n_tau: int
    n_spin: int
    beta: float
    nk: tuple = (1, 1, 1)
    tau: np.ndarray = None
    G: np.ndarray = None
    X: np.ndarray = None
    V: np.ndarray = None
    extras: dict = field(default_factory=dict)

    @property
    def n_k(self) -> int:
        return int(np.prod(self.nk))

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.G)


def molecule(cfg: int, n: int, N: int, n_tau: int, beta: float, n_spin: int = 1,
             spin_shift: float = 0.05, shift_orbitals: int = 10, instance: int | None = None,
             name: str | None = None) -> Workload:
    """Molecule-like instance (1 k-point, real data)."""
    h, e, u = random_hamiltonian(_rng(cfg, 0, instance), n)
    mu = half_filling_mu(e)
    tau = tau_nodes(n_tau, beta)
    if n_spin == 1:
        G = green_tau(e, u, mu, tau, beta)[None, None]
    else:
        m = min(shift_orbitals, n)
        Gs = []
        for sgn in (-1.0, 1.0):
            hs = h.copy()
            hs[np.arange(m), np.arange(m)] += sgn * spin_shift
            es, us = np.linalg.eigh(hs)
            Gs.append(green_tau(es, us, mu, tau, beta))
        G = np.stack(Gs)[:, None]
    X = (_rng(cfg, 1, instance).standard_normal((N, n)) / np.sqrt(n))[None]
    z = decaying_metric(_rng(cfg, 2, instance), N)
    V = (z @ z.T)[None]
    return Workload(name or f"molecule-c{cfg}", n, N, n_tau, n_spin, beta, (1, 1, 1), tau,
                    np.ascontiguousarray(G), np.ascontiguousarray(X), np.ascontiguousarray(V),
                    {"mu": mu, "eps": e, "U": u})


def config(c: int) -> Workload:
    """The five stand-in workloads (molecule c0..c2, solid c3; c4 see ``batch_c4``)."""
    if c == 0:
        return molecule(0, 20, 80, 30, 100.0, 1, name="sox-c0-n20-N80-t30")
    if c == 1:
        return molecule(1, 120, 600, 80, 100.0, 2, name="sox-c1-n120-N600-t80-uhf")
    if c == 2:
        return molecule(2, 250, 2000, 100, 100.0, 1, name="sosex-c2-n250-N2000-t100")
    if c == 3:
        return solid(3, (3, 3, 3), 26, 300, 60, 300.0, name="sosexdyn-c3-k333-n26-N300-t60")
    raise ValueError(f"config {c} has no single-instance form; use batch_c4()")


def batch_c4_sizes() -> np.ndarray:
    return _rng(4, 4).integers(40, 401, size=16)


def batch_c4(max_instances: int | None = None) -> list[Workload]:
    """16 uneven instances, n ~ U{40..400}, N = 6n, 120 tau, beta = 100."""
    sizes = batch_c4_sizes()
    if max_instances is not None:
        sizes = sizes[:max_instances]
    return [c4_instance(i) for i in range(len(sizes))]


def bosonic_transforms(tau: np.ndarray, beta: float, M: int, n_gl: int = 512):
    """Caller-side tau <-> i Omega transform pair for bosonic functions on the grid.

    Omega_m = 2 pi m / beta, m = -M..M.  T_fwd[m][j] = int_0^beta e^{i Omega_m s} L_j(s) ds with
    L_j the cardinal polynomial of the Chebyshev-Lobatto nodes (barycentric form), integrated
    by n_gl-point Gauss-Legendre; T_inv[i][m] = e^{-i Omega_m tau_i} / beta.  These are inputs
    (the paper takes its grids and transforms from sparse-ir), not self-energy arithmetic.
    """
    n = tau.size
    om = 2.0 * np.pi * np.arange(-M, M + 1) / beta
    x, wg = np.polynomial.legendre.leggauss(n_gl)
    s = 0.5 * beta * (x + 1.0)
    wg = 0.5 * beta * wg
    bw = np.array([(-1.0) ** j for j in range(n)])
    bw[0] *= 0.5
    bw[-1] *= 0.5
    d = s[:, None] - tau[None, :]
    ratio = bw[None, :] / d
    L = ratio / ratio.sum(axis=1, keepdims=True)          # [gl][j]
    T_fwd = (np.exp(1j * om[:, None] * s[None, :]) * wg[None, :]) @ L
    T_inv = np.exp(-1j * tau[:, None] * om[None, :]) / beta
    return om, np.ascontiguousarray(T_fwd), np.ascontiguousarray(T_inv)


def fermionic_transform(tau: np.ndarray, beta: float, n_max: int, n_gl: int = 16):
    """Caller-side tau -> i w transform for fermionic functions on the grid.

    w_m = (2m+1) pi / beta, m = -n_max .. n_max-1.  T_w[m][j] = int_0^beta e^{i w_m s} L_j(s) ds
    with L_j the cardinal polynomial of the Chebyshev-Lobatto nodes (barycentric form),
    integrated by composite n_gl-point Gauss-Legendre with at least two panels per period of
    the highest frequency.  An input of the loop's frequency transform (the paper takes its
    grids and transforms from sparse-ir), not self-energy arithmetic.  Returns (w, T_w)."""
    n = tau.size
    m = np.arange(-n_max, n_max)
    om = (2 * m + 1) * np.pi / beta
    n_pan = max(8, int(np.ceil(np.abs(om).max() * beta / np.pi)) + 1)
    x, wg = np.polynomial.legendre.leggauss(n_gl)
    edges = np.linspace(0.0, beta, n_pan + 1)
    half = 0.5 * np.diff(edges)
    s = (edges[:-1, None] + half[:, None] * (x[None, :] + 1.0)).ravel()
    ws = (half[:, None] * wg[None, :]).ravel()
    bw = np.array([(-1.0) ** j for j in range(n)])
    bw[0] *= 0.5
    bw[-1] *= 0.5
    d = s[:, None] - tau[None, :]
    exact = np.abs(d) < 1e-300
    d = np.where(exact, 1.0, d)
    ratio = bw[None, :] / d
    L = ratio / ratio.sum(axis=1, keepdims=True)
    rows = exact.any(axis=1)
    L[rows] = exact[rows].astype(float)
    T_w = np.empty((om.size, n), complex)
    for a in range(0, om.size, 64):
        T_w[a:a + 64] = (np.exp(1j * om[a:a + 64, None] * s[None, :]) * ws[None, :]) @ L
    return om, np.ascontiguousarray(T_w)


def c4_instance(i: int) -> Workload:
    """Instance i of the uneven batch (n from the batch-size stream, N = 6n, 120 tau)."""
    n = int(batch_c4_sizes()[i])
    return molecule(4, n, 6 * n, 120, 100.0, 1, instance=i, name=f"c4-inst{i}-n{n}")


def c4_smallest(k: int = 3) -> list[int]:
    """Indices of the k smallest instances of the uneven batch."""
    return [int(i) for i in np.argsort(batch_c4_sizes(), kind="stable")[:k]]


def kmesh(nk: tuple) -> np.ndarray:
    """Integer k labels m in [0, nk_d) for each direction, k = 2 pi m / nk (row-major order)."""
    g = np.stack(np.meshgrid(*[np.arange(d) for d in nk], indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def kindex(m: np.ndarray, nk: tuple) -> int:
    m = np.mod(m, nk)
    return int((m[0] * nk[1] + m[1]) * nk[2] + m[2])


def solid(cfg: int, nk: tuple, n: int, N: int, n_tau: int, beta: float,
          hop: float = 0.1, name: str | None = None) -> Workload:
    """Periodic stand-in: tight-binding H0(k), complex X^k with Bloch phases, V^q Hermitian PSD."""
    ks = kmesh(nk)
    nkt = ks.shape[0]
    h_on, _, _ = random_hamiltonian(_rng(cfg, 0), n)
    rx = _rng(cfg, 3)
    T = [rx.standard_normal((n, n)) * hop / np.sqrt(n) for _ in range(3)]
    kvec = 2.0 * np.pi * ks / np.asarray(nk)[None, :]
    Hk = np.empty((nkt, n, n), complex)
    for ik in range(nkt):
        H = h_on.astype(complex)
        for d in range(3):
            ph = np.exp(1j * kvec[ik, d])
            H = H + T[d] * ph + T[d].T * np.conj(ph)
        Hk[ik] = 0.5 * (H + H.conj().T)
    evals, evecs = np.linalg.eigh(Hk)
    # chemical potential by bisection to half filling at this beta
    target = 0.5 * n * nkt
    lo, hi = float(evals.min()) - 1.0, float(evals.max()) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        x = np.clip(beta * (evals - mid), -700, 700)
        cnt = np.sum(1.0 / (1.0 + np.exp(x)))
        lo, hi = (mid, hi) if cnt < target else (lo, mid)
    mu = 0.5 * (lo + hi)
    tau = tau_nodes(n_tau, beta)
    G = np.stack([green_tau(evals[ik], evecs[ik], mu, tau, beta) for ik in range(nkt)])[None]
    rxp = _rng(cfg, 1)
    x0 = (rxp.standard_normal((N, n)) + 1j * rxp.standard_normal((N, n))) / np.sqrt(2.0 * n)
    rP = rxp.random((N, 3))
    X = np.stack([x0 * np.exp(1j * (rP @ kvec[ik]))[:, None] for ik in range(nkt)])
    # V^q = Z^q Z^q^H with V^{-q} = conj(V^q); q = 0 real
    rz = _rng(cfg, 2)
    V = np.empty((nkt, N, N), complex)
    done = np.zeros(nkt, bool)
    for iq in range(nkt):
        if done[iq]:
            continue
        jq = kindex(-ks[iq], nk)
        z = decaying_metric(rz, N, complex_=(jq != iq))
        vq = z @ z.conj().T
        V[iq] = vq
        V[jq] = vq.conj()
        done[iq] = done[jq] = True
    return Workload(name or f"solid-c{cfg}", n, N, n_tau, 1, beta, tuple(nk), tau,
                    np.ascontiguousarray(G), np.ascontiguousarray(X), np.ascontiguousarray(V),
                    {"mu": mu, "eps": evals, "U": evecs, "kvec": kvec, "r_P": rP})


def tiny(n: int, N: int, n_tau: int = 6, beta: float = 4.0, n_spin: int = 1, seed: int = 7) -> Workload:
    """Small random molecule-like case for unit tests (same recipe, free seed)."""
    w = molecule(100 + seed, n, N, n_tau, beta, n_spin, name=f"tiny-n{n}-N{N}-t{n_tau}-s{seed}")
    return w


def pole_screening(V: np.ndarray, beta: float, M: int, omega_p: float = 0.5, strength: float = 0.5,
                   seed: int = 0) -> np.ndarray:
    """Synthetic dynamic screening W_d^q(i Omega_m), m = -M..M, for timing runs.

    A single-pole stand-in with the structure of W - v (no RPA is evaluated here):
    W_d^q(i Omega) = -strength * omega_p^2 / (Omega^2 + omega_p^2) * V^q D V^q / ||V^0||,
    D a seeded positive diagonal.  Hermitian and even in Omega per q, and
    W_d^{-q} = conj(W_d^q) whenever V^{-q} = conj(V^q).  Shape [n_q][2M+1][N][N].
    """
    rng = np.random.default_rng([2412188290, 7, seed])
    nq, N, _ = V.shape
    d = rng.uniform(0.5, 1.5, size=N)
    norm = float(np.linalg.norm(V[0], 2))
    om = 2.0 * np.pi * np.arange(-M, M + 1) / beta
    f = -strength * omega_p ** 2 / (om ** 2 + omega_p ** 2) / norm
    out = np.empty((nq, 2 * M + 1, N, N), dtype=np.result_type(V, np.float64))
    for q in range(nq):
        vdv = (V[q] * d[None, :]) @ V[q]
        vdv = 0.5 * (vdv + vdv.conj().T)
        for m in range(2 * M + 1):
            out[q, m] = f[m] * vdv
    return out
