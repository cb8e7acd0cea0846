"""Plain FP64 CPU oracle of the regularized fluctuating lattice Boltzmann step (Reg-FLBM,
D3Q27) of Lauricella, Montessori, Tiribocchi and Succi, arXiv 2507.08820.

TEST INFRASTRUCTURE ONLY. This module is the correctness reference for the CUDA
library. Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it; the library never calls it, and it shares no code, table or helper with the
CUDA sources. Every array is float64; the per-site algebra follows the paper's equations
in their order, with naive loops and dense 27x27 products and no factorisation.

Equation numbers are the paper's numbered equations in order of appearance:
  Eq. 1 BGK LBE, Eq. 2 second-order equilibrium, Eqs. 3-4 density and momentum,
  Eq. 5 moments, Eq. 6 norms b_k, Eq. 7 collision, Eq. 8 streaming, Eq. 9 relaxed
  non-equilibrium moments plus noise, Eq. 10 noise amplitude, Eq. 11 back transform,
  Eq. 12 BGK-FLBM, Eqs. 17-18 Hermite expansions, Eqs. 19-20 Hermite projections,
  Eq. 21 recursive equilibrium coefficients, Eq. 22 recursive non-equilibrium
  coefficients, Eq. 23 b_k from order and multiplicity, Eq. 24 Reg-FLBM,
  Eq. 25 Reg-FLBM with hydrodynamic/ghost split, Eqs. 26-27 equilibrium and
  hydrodynamic non-equilibrium parts.

Readings taken where the paper is silent or ambiguous (each listed in the design notes):
  * velocity order inside the groups of Table I (see `velocities`);
  * the generator of the standard normals r_k (Sec. II.A names none): Philox4x32-10
    (Salmon et al., SC'11) with counter (site, step, call j, replica) and key
    (seed low 32 bits, seed high 32 bits); uniforms (x + 1/2) 2^-32; Box-Muller pairs;
    r_k = n[k - 4] for k = 4..26 from the 24 normals n of calls j = 0..5;
  * rho in Eq. 10 is the local density of the site (option: the reference rho0);
  * Eq. 22's "perm" is the sum over the first n-1 indices paired with the last one;
  * the equilibrium of Eq. 26 uses the coefficients of Eq. 21 (the text points at
    Eq. 22, which is the non-equilibrium recursion);
  * Pi (Sec. III) is the second Hermite coefficient a^(2) = sum_i f_i H^(2)_i;
  * a thermal initial state (`thermal_state`): independent Gaussian modes with the
    variances Eq. 10 maintains, drawn with Philox calls j = 6..12 of step 0.

Layout: populations are arrays of shape (27, N) for N = nx*ny*nz sites with site index
s = x + nx*(y + ny*z); the state held between steps is the pre-collision f(x, t).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

Q = 27
CS2 = 1.0 / 3.0          # c_s^2 in lattice units (Sec. II.A, below Eq. 1)
AXES = "xyz"


# --------------------------------------------------------------------------- Table I
def velocities() -> np.ndarray:
    """D3Q27 velocities c_i, shape (27, 3), int (Table I).

    Table I fixes only the groups i = 0, 1-6, 7-18, 19-26. Order inside the groups
    (reading): 1..6 = +x, -x, +y, -y, +z, -z; 7..18 = the (x,y), then (x,z), then (y,z)
    diagonals, each as (+,+), (+,-), (-,+), (-,-); 19..26 = (+-1, +-1, +-1) counting in
    binary with x slowest and + before -.
    """
    c = [(0, 0, 0)]
    for axis in range(3):
        for sign in (1, -1):
            v = [0, 0, 0]
            v[axis] = sign
            c.append(tuple(v))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        for sa, sb in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            v = [0, 0, 0]
            v[a], v[b] = sa, sb
            c.append(tuple(v))
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                c.append((sx, sy, sz))
    return np.array(c, dtype=np.int64)


def weights(c: np.ndarray | None = None) -> np.ndarray:
    """Lattice weights w_i by |c_i|^2 (Table I): 8/27, 2/27, 1/54, 1/216."""
    c = velocities() if c is None else c
    by_norm = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}
    return np.array([by_norm[int(v @ v)] for v in c])


def opposite(c: np.ndarray | None = None) -> np.ndarray:
    """Index of -c_i for every i."""
    c = velocities() if c is None else c
    return np.array([int(np.flatnonzero((c == -v).all(axis=1))[0]) for v in c])


# -------------------------------------------------------------------------- Table II
# Each mode k: its Hermite index sequence (the subscript of H^(n) in Table II, with
# x^2 written xx), its order n_k and multiplicity mu_k, and the polynomial e_ki of
# Table II written out term by term.
_S = CS2


def _modes():
    return [
        ("", 0, 1, lambda x, y, z: np.ones_like(x)),
        ("x", 1, 1, lambda x, y, z: x),
        ("y", 1, 1, lambda x, y, z: y),
        ("z", 1, 1, lambda x, y, z: z),
        ("xx", 2, 1, lambda x, y, z: x * x - _S),
        ("yy", 2, 1, lambda x, y, z: y * y - _S),
        ("zz", 2, 1, lambda x, y, z: z * z - _S),
        ("xy", 2, 2, lambda x, y, z: x * y),
        ("xz", 2, 2, lambda x, y, z: x * z),
        ("yz", 2, 2, lambda x, y, z: y * z),
        ("xxy", 3, 3, lambda x, y, z: x * x * y - _S * y),
        ("xxz", 3, 3, lambda x, y, z: x * x * z - _S * z),
        ("xyy", 3, 3, lambda x, y, z: x * y * y - _S * x),
        ("xzz", 3, 3, lambda x, y, z: x * z * z - _S * x),
        ("yzz", 3, 3, lambda x, y, z: y * z * z - _S * y),
        ("yyz", 3, 3, lambda x, y, z: y * y * z - _S * z),
        ("xyz", 3, 6, lambda x, y, z: x * y * z),
        ("xxyy", 4, 6, lambda x, y, z: x * x * y * y - _S * (x * x + y * y) + _S ** 2),
        ("xxzz", 4, 6, lambda x, y, z: x * x * z * z - _S * (x * x + z * z) + _S ** 2),
        ("yyzz", 4, 6, lambda x, y, z: y * y * z * z - _S * (y * y + z * z) + _S ** 2),
        ("xyzz", 4, 12, lambda x, y, z: x * y * z * z - _S * x * y),
        ("xyyz", 4, 12, lambda x, y, z: x * y * y * z - _S * x * z),
        ("xxyz", 4, 12, lambda x, y, z: x * x * y * z - _S * y * z),
        ("xxyzz", 5, 30, lambda x, y, z: x * x * y * z * z
         - _S * (x * x * y + y * z * z) + _S ** 2 * y),
        ("xxyyz", 5, 30, lambda x, y, z: x * x * y * y * z
         - _S * (x * x * z + y * y * z) + _S ** 2 * z),
        ("xyyzz", 5, 30, lambda x, y, z: x * y * y * z * z
         - _S * (x * y * y + x * z * z) + _S ** 2 * x),
        ("xxyyzz", 6, 90, lambda x, y, z: x * x * y * y * z * z
         - _S * (x * x * y * y + x * x * z * z + y * y * z * z)
         + _S ** 2 * (x * x + y * y + z * z) - _S ** 3),
    ]


MODE_SEQ = tuple(m[0] for m in _modes())          # Hermite index sequence of mode k
MODE_ORDER = np.array([m[1] for m in _modes()])   # n_k
MODE_MULT = np.array([m[2] for m in _modes()])    # mu_k
HYDRO = tuple(range(4, 10))                       # non-conserved hydrodynamic modes
GHOST = tuple(range(10, 27))                      # ghost modes


def basis(c: np.ndarray | None = None) -> np.ndarray:
    """E[k, i] = e_ki of Table II evaluated on the velocities, shape (27, 27)."""
    c = (velocities() if c is None else c).astype(np.float64)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    return np.array([poly(x, y, z) for (_, _, _, poly) in _modes()])


def norms(E: np.ndarray | None = None, w: np.ndarray | None = None) -> np.ndarray:
    """b_k = sum_i w_i e_ki^2 (Eq. 6)."""
    E = basis() if E is None else E
    w = weights() if w is None else w
    return (E * E) @ w


# ----------------------------------------------------------------- moments (Eqs. 3-5)
def density(f: np.ndarray) -> np.ndarray:
    """rho = sum_i f_i (Eq. 3)."""
    return f.sum(axis=0)


def momentum(f: np.ndarray) -> np.ndarray:
    """rho u_alpha = sum_i f_i c_i,alpha (Eq. 4), shape (3, N)."""
    return velocities().T.astype(np.float64) @ f


def moments(f: np.ndarray) -> np.ndarray:
    """m_k = sum_i e_ki f_i (Eq. 5), shape (27, N)."""
    return basis() @ f


def back_transform(m: np.ndarray) -> np.ndarray:
    """f_i = w_i sum_k b_k^-1 e_ki m_k (Eq. 11)."""
    E, w = basis(), weights()
    b = norms(E, w)
    return w[:, None] * (E.T @ (m / b[:, None]))


# ----------------------------------------------------- Hermite coefficients (Eqs. 19-22)
def a0_coefficient(seq: str, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Equilibrium Hermite coefficient a_0^(n) for the index sequence seq by the
    recursion of Eq. 21: a_0^(0) = rho and a_0^(n) = a_0^(n-1) u_(alpha_n)."""
    if seq == "":
        return rho.copy()
    return a0_coefficient(seq[:-1], rho, u) * u[AXES.index(seq[-1])]


def a1_coefficient(seq: str, a1_2: dict, u: np.ndarray) -> np.ndarray:
    """Non-equilibrium Hermite coefficient a_1^(n), n >= 2, by the recursion of Eq. 22.

    a1_2 maps an ordered pair of axes (alpha, beta) to a_1^(2)_(alpha beta) (Eq. 20).
    For n >= 3: a_1^(n) = a_1^(n-1)[first n-1 indices] u_(alpha_n) plus, for each of the
    first n-1 indices alpha_l, a_1^(2)_(alpha_l alpha_n) times the product of u over the
    other n-2 of the first n-1 indices (the "perm" term of Eq. 22).
    """
    n = len(seq)
    if n < 2:
        raise ValueError("a_1^(n) is defined for n >= 2 only (Eq. 20)")
    if n == 2:
        return a1_2[(seq[0], seq[1])]
    last = seq[-1]
    out = a1_coefficient(seq[:-1], a1_2, u) * u[AXES.index(last)]
    for l in range(n - 1):
        term = a1_2[(seq[l], last)].copy()
        for m in range(n - 1):
            if m != l:
                term = term * u[AXES.index(seq[m])]
        out = out + term
    return out


def hermite_equilibrium(rho: np.ndarray, u: np.ndarray, max_order: int = 6) -> np.ndarray:
    """f_i^(0) = w_i sum_k mu_k / (c_s^(2 n_k) n_k!) a_0,k H_k,i (Eq. 26) over the modes
    with n_k <= max_order (max_order = 6 is the full D3Q27 expansion used by both models,
    Sec. III; max_order = 2 is the truncation that Sec. II.B equates with Eq. 2)."""
    E, w = basis(), weights()
    # the sum over k written as one product: sum_k E[k, i] (weight_k a_0,k)
    coef = np.array([_expansion_weight(k) if MODE_ORDER[k] <= max_order else 0.0
                     for k in range(Q)])
    a0 = np.array([a0_coefficient(seq, rho, u) for seq in MODE_SEQ])
    return w[:, None] * (E.T @ (coef[:, None] * a0))


def _expansion_weight(k: int) -> float:
    """mu_k / (c_s^(2 n_k) n_k!), the weight of mode k in Eqs. 26-27."""
    n = int(MODE_ORDER[k])
    return MODE_MULT[k] / (CS2 ** n * math.factorial(n))


def second_order_equilibrium(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """The classic equilibrium of Eq. 2 (used only as a reference identity)."""
    c, w = velocities().astype(np.float64), weights()
    cu = c @ u
    uu = (u * u).sum(axis=0)
    return w[:, None] * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 ** 2) - uu / (2 * CS2))


def hermite_a2(f: np.ndarray) -> np.ndarray:
    """Pi_ab = a^(2)_ab = sum_i f_i H^(2)_ab,i (Eqs. 19-20 summed; Sec. III), rows
    xx, yy, zz, xy, xz, yz (the modes k = 4..9 of Table II)."""
    return moments(f)[4:10]


# ----------------------------------------------------------------- noise (Eq. 9-10)
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57     # Salmon et al. (SC'11), Philox4x32
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85     # Weyl key increments
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).

    ctr: four arrays (or ints) of uint32 counter words; key: two uint32 key words.
    One round maps (c0, c1, c2, c3) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
    hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by the Weyl constants between
    rounds. Returns four uint64 arrays holding uint32 values.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _MASK)
        k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
        k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
    return c0, c1, c2, c3


def uniform01(x):
    """uint32 -> (x + 1/2) 2^-32 in (0, 1)."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(x0, x1):
    """Two uint32 draws -> two independent standard normals (Box and Muller, 1958):
    sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1)."""
    r = np.sqrt(-2.0 * np.log(uniform01(x0)))
    t = 2.0 * np.pi * uniform01(x1)
    return r * np.cos(t), r * np.sin(t)


def normals(seed: int, step: int, sites, replica: int = 0) -> np.ndarray:
    """The 24 standard normals n[0..23] of every site at one step, shape (24, M).

    Call j = 0..5 draws Philox4x32-10 at counter (site, step, j, replica) and key
    (seed mod 2^32, seed div 2^32); its words (x0, x1) and (x2, x3) give the Box-Muller
    pairs n[4j], n[4j+1] and n[4j+2], n[4j+3].
    """
    sites = np.asarray(sites, dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((24, sites.size))
    for j in range(6):
        x0, x1, x2, x3 = philox4x32_10(
            (sites, np.full_like(sites, step & 0xFFFFFFFF), np.full_like(sites, j),
             np.full_like(sites, replica)), key)
        out[4 * j], out[4 * j + 1] = box_muller(x0, x1)
        out[4 * j + 2], out[4 * j + 3] = box_muller(x2, x3)
    return out


def noise_amplitude(rho, kT: float, omega_k: float, b_k: float):
    """phi_k = sqrt(rho kT omega_k (2 - omega_k) b_k / c_s^2) (Eq. 10)."""
    return np.sqrt(rho * kT * omega_k * (2.0 - omega_k) * b_k / CS2)


# --------------------------------------------------------------------- collision
def collide(f, tau: float, kT: float, seed: int, step: int, sites, replica: int = 0,
            omega_g: float = 1.0, model: str = "reg", rho0: float = 1.0,
            phi_rho: str = "local", r=None):
    """Post-collision populations f* at every site of f, shape (27, M).

    model = "reg": Reg-FLBM, Eq. 25 (with Eq. 24's ghost term kept for omega_g != 1):
      f* = f^(0) + (1 - omega_h) f^(1,h) + (1 - omega_g) f^(1,g)
           + w_i sum_{k=4..26} b_k^-1 e_ki phi_k r_k,
    with f^(0) from Eq. 26 (coefficients of Eq. 21), f^(1,h) from Eq. 27 with
    a_1^(2) = m - a_0^(2) (Eq. 20 with f^(1) = f - f^(0), Eq. 15), f^(1,g) the same sum
    over k = 10..26 with the coefficients of Eq. 22, omega_h = 1/tau, and phi_k of
    Eq. 10 evaluated with omega_h for k = 4..9 and omega_g for k = 10..26.
    model = "bgk": BGK-FLBM, Eq. 12, with f^eq = f^(0) of Eq. 26 (Sec. III):
      f* = f^(0) + (1 - omega)(f - f^(0)) + w_i sum_{k=4..26} b_k^-1 e_ki phi_k r_k.
    r: optional (23, M) normals r_4..r_26; drawn by `normals` when None.
    """
    E, w = basis(), weights()
    b = norms(E, w)
    omega_h = 1.0 / tau
    rho = density(f)
    u = momentum(f) / rho
    m = E @ f

    f0 = hermite_equilibrium(rho, u)
    if r is None:
        r = normals(seed, step, sites, replica)[:23]
    phi_rho = rho if phi_rho == "local" else np.full_like(rho, rho0)

    if model == "bgk":
        fstar = f0 + (1.0 - omega_h) * (f - f0)
        omega_of = lambda k: omega_h
    elif model == "reg":
        a0 = np.array([a0_coefficient(seq, rho, u) for seq in MODE_SEQ])
        a1_2 = {}
        for k in HYDRO:
            a, bb = MODE_SEQ[k]
            a1_2[(a, bb)] = m[k] - a0[k]
            a1_2[(bb, a)] = a1_2[(a, bb)]
        # Eq. 27: f^(1,h)_i = w_i sum_{k=4..9} weight_k a_1,k H_k,i
        a1h = np.array([_expansion_weight(k) * a1_2[tuple(MODE_SEQ[k])] for k in HYDRO])
        f1h = w[:, None] * (E[4:10].T @ a1h)
        fstar = f0 + (1.0 - omega_h) * f1h
        if omega_g != 1.0:
            # the ghost part of Eq. 24's split, coefficients from Eq. 22
            a1g = np.array([_expansion_weight(k) * a1_coefficient(MODE_SEQ[k], a1_2, u)
                            for k in GHOST])
            f1g = w[:, None] * (E[10:].T @ a1g)
            fstar = fstar + (1.0 - omega_g) * f1g
        omega_of = lambda k: omega_h if k in HYDRO else omega_g
    else:
        raise ValueError(model)

    if kT > 0.0:
        # w_i sum_{k=4..26} b_k^-1 e_ki phi_k r_k
        phr = np.array([noise_amplitude(phi_rho, kT, omega_of(k), b[k]) * r[k - 4] / b[k]
                        for k in range(4, 27)])
        fstar = fstar + w[:, None] * (E[4:].T @ phr)
    return fstar


# --------------------------------------------------------------------- streaming
def stream(fstar: np.ndarray, shape) -> np.ndarray:
    """f_i(x + c_i, t + 1) = f*_i(x, t) on a periodic box (Eq. 8)."""
    nx, ny, nz = shape
    c = velocities()
    out = np.empty_like(fstar)
    for i in range(Q):
        plane = fstar[i].reshape(nz, ny, nx)
        out[i] = np.roll(plane, shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)).ravel()
    return out


def step(f, shape, tau: float, kT: float, seed: int, t: int, replica: int = 0, **kw):
    """One time step t -> t + 1 of the whole box: collision at every site (noise keyed by
    the site index and t) followed by periodic streaming. Returns f(x, t + 1)."""
    sites = np.arange(f.shape[1], dtype=np.uint64)
    return stream(collide(f, tau, kT, seed, t, sites, replica, **kw), shape)


def run(f, shape, tau, kT, seed, steps, t0=0, replica=0, **kw):
    """`steps` successive steps starting at step index t0."""
    for t in range(t0, t0 + steps):
        f = step(f, shape, tau, kT, seed, t, replica, **kw)
    return f


# --------------------------------------------------------------- initial states
def rest_state(n_sites: int, rho0: float = 1.0) -> np.ndarray:
    """Fluid at rest: f_i = w_i rho0 (Eq. 26 at u = 0)."""
    return np.outer(weights(), np.full(n_sites, rho0))


def equilibrium_state(rho, u) -> np.ndarray:
    """f_i = f_i^(0)(rho, u) (Eq. 26) at every site."""
    return hermite_equilibrium(np.asarray(rho, float), np.asarray(u, float))


def macroscopic(f):
    """(rho, u, Pi) at every site: Eqs. 3-4 and Pi = a^(2) (Sec. III)."""
    rho = density(f)
    return rho, momentum(f) / rho, hermite_a2(f)


@lru_cache(maxsize=None)
def _tables_cached():
    E, w = basis(), weights()
    return E, w, norms(E, w)


def thermal_state(kT: float, seed: int, sites, rho0: float = 1.0, replica: int = 0) -> np.ndarray:
    """A draw from the stationary distribution of the linearised fluctuating model: at
    every site all 27 modes m_k of Table II (density and momentum included) are
    independent normals of variance rho0 kT b_k / c_s^2, the per-mode variance that the
    amplitude of Eq. 10 maintains (Sec. II.A, after Eq. 10), around the rest state:
    f = w rho0 + back_transform(m) (Eq. 11). Shape (27, M).

    Noise words (a reading; the paper starts from rest): Philox4x32-10 calls j = 6..12 at
    counter (site, 0, j, replica) and key (seed mod 2^32, seed div 2^32), outside the calls
    j = 0..5 of the steps; Box-Muller pairs in order give n[0..27]; m_k = sqrt(rho0 kT b_k
    / c_s^2) n[k] for k = 0..26.
    """
    sites = np.asarray(sites, dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    n = np.empty((28, sites.size))
    for j in range(7):
        x0, x1, x2, x3 = philox4x32_10(
            (sites, np.zeros_like(sites), np.full_like(sites, 6 + j), np.full_like(sites, replica)), key)
        n[4 * j], n[4 * j + 1] = box_muller(x0, x1)
        n[4 * j + 2], n[4 * j + 3] = box_muller(x2, x3)
    m = np.sqrt(fdt_mode_variance(rho0, kT))[:, None] * n[:Q]
    return rest_state(sites.size, rho0) + back_transform(m)


def fdt_mode_variance(rho0: float, kT: float) -> np.ndarray:
    """Equilibrium variance of every mode per site, rho0 kT b_k / c_s^2: the variance
    the amplitude of Eq. 10 is built to sustain (Sec. II.A, after Eq. 10)."""
    _, _, b = _tables_cached()
    return rho0 * kT * b / CS2
