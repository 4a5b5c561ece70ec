"""CPU FP64 oracle for the direction-restricted periodized DVM operator.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the CUDA implementation in ``paper_1201_3986_gb300``; the two meet only
through the seeded inputs of ``synth``.

The arithmetic lives in ``qdvm_oracle.c`` (plain C, FP64, Neumaier
compensated sums, OpenMP over output points); this module compiles it with
gcc on first use and marshals numpy arrays.

Functions and the passages they follow:

* ``lines(d, m)``            -- the line sets A^1 / A^2 of Section 3.2 (brute
  force over [-m, m]^d).
* ``q(...)`` / ``q_points``  -- eq. (DR) of Section 2.3 with the decoupled
  weights of eq. (decoup) and the line restriction of eq. (decDVM).
* ``jvp`` / ``vjp``          -- derivative of that quadratic form and the
  transpose of its Jacobian (scattered term by term); ``jvp_points`` /
  ``vjp_points`` the same at selected points (the VJP as a gather).
* ``moments``                -- mass, momentum and energy of Section 2.1.
* ``dtr(...)``               -- the box-truncated operator D^tr of Section
  2.3 (the same terms, counted only when all four velocities lie in the
  grid): exactly conservative, not a convolution.
* ``equilibrium_distance``   -- the distance of a cell to the Maxwellian
  with its own discrete moments, the indicator for a space-dependent Nbar
  (Section 3.3 leaves the indicator open; this is the reading used).
* ``rk2(...)``               -- the second-order TVD Runge-Kutta time
  stepping of Section 4 for df/dt = Q(f) (Shu-Osher form), in numpy around
  ``q``.
* ``default_ntilde(N)``      -- Ntilde = floor(N / (3 + sqrt 2)), Section 4.
* ``spectral_beta(...)`` / ``q_spectral(...)`` -- the pseudo-spectral form
  of Section 3.1: the kernel modes beta(K, L) of eq. (betaKL) summed term by
  term over the (k, l) pairs, beta~(K, L) = beta(K, L) - beta(L, L), and
  Q through eq. (sysDiff) with numpy's FFT (small grids only: the table
  has N^{2d} entries).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute force through the general DVM form of
eq. (TypicalDVM), and the Fourier-side formula of eq. (sysDiff)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdvm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNELS = {"unit": 0, "hp": 1}


def build(force: bool = False) -> str:
    """Compile qdvm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True)
    except (subprocess.CalledProcessError, FileNotFoundError):
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dbl_p = P(ctypes.c_double)
        i64_p = P(ctypes.c_int64)
        lib.oracle_default_ntilde.argtypes = [ctypes.c_int]
        lib.oracle_default_ntilde.restype = ctypes.c_int
        lib.oracle_lines.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int]
        lib.oracle_lines.restype = ctypes.c_int
        lib.oracle_terms_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_terms_count.restype = ctypes.c_int
        lib.oracle_q_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, dbl_p, i64_p, ctypes.c_int64, dbl_p, dbl_p, dbl_p, dbl_p]
        lib.oracle_q_points.restype = ctypes.c_int
        lib.oracle_dtr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, dbl_p, dbl_p, dbl_p]
        lib.oracle_dtr.restype = ctypes.c_int
        for name in ("oracle_jvp", "oracle_vjp"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_double, dbl_p, dbl_p, dbl_p]
            fn.restype = ctypes.c_int
        lib.oracle_vjp_scale.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, dbl_p, dbl_p, dbl_p, dbl_p]
        lib.oracle_vjp_scale.restype = ctypes.c_int
        for name in ("oracle_jvp_points", "oracle_vjp_points"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_double, dbl_p, dbl_p, i64_p, ctypes.c_int64, dbl_p, dbl_p]
            fn.restype = ctypes.c_int
        lib.oracle_moments.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dbl_p, dbl_p]
        lib.oracle_moments.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_ntilde(N: int) -> int:
    return int(_load().oracle_default_ntilde(int(N)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def lines(d: int, m: int) -> np.ndarray:
    """Primitive directions of [-m, m]^d up to sign, shape (count, d), ordered
    by |e|_inf then lexicographically."""
    lib = _load()
    n = lib.oracle_lines(d, m, None, 0)
    out = np.zeros((max(n, 1), d), dtype=np.int32)
    lib.oracle_lines(d, m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n)
    return out[:n]


def terms_count(d: int, Ntilde: int, m: int) -> int:
    return int(_load().oracle_terms_count(d, Ntilde, m))


def _params(f: np.ndarray, L: float, Nbar: int, Ntilde: int | None):
    d = f.ndim
    N = f.shape[0]
    if any(s != N for s in f.shape):
        raise ValueError("f must be N^d")
    Nt = default_ntilde(N) if Ntilde is None else int(Ntilde)
    m = min(int(Nbar), Nt)
    h = 2.0 * L / N
    return d, N, Nt, m, h


def q_points(f, L: float, Nbar: int, idx=None, kernel: str = "unit", Ntilde: int | None = None) -> dict:
    """Q, gain, loss and scale = sum of |terms| at flat indices ``idx`` (all
    points when None)."""
    f = _f64(f)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    if idx is None:
        n = f.size
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n = idx.size
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    Q, G, Lo, S = (np.zeros(n) for _ in range(4))
    rc = _load().oracle_q_points(d, N, Nt, m, KERNELS[kernel], h, _dp(f), ip, n, _dp(Q), _dp(G), _dp(Lo), _dp(S))
    if rc != 0:
        raise RuntimeError(f"oracle_q_points failed ({rc})")
    if idx is None:
        Q, G, Lo, S = (a.reshape(f.shape) for a in (Q, G, Lo, S))
    return {"Q": Q, "gain": G, "loss": Lo, "scale": S}


def q(f, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None) -> dict:
    return q_points(f, L, Nbar, None, kernel, Ntilde)


def dtr(f, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None) -> dict:
    """The box-truncated operator D^tr of Section 2.3 with the terms of ``q``:
    no periodisation, a term counts only when its four velocities lie in
    the grid.  Returns Q and scale = sum of |terms|."""
    f = _f64(f)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    Q, sc = np.zeros_like(f), np.zeros_like(f)
    rc = _load().oracle_dtr(d, N, Nt, m, KERNELS[kernel], h, _dp(f), _dp(Q), _dp(sc))
    if rc != 0:
        raise RuntimeError(f"oracle_dtr failed ({rc})")
    return {"Q": Q, "scale": sc}


def equilibrium_distance(f, L: float) -> float:
    """sum |f - M| / sum |f| with M the Maxwellian of the discrete moments
    rho = h^d sum f, u = h^d sum f v / rho, T = (h^d sum f |v|^2 / rho -
    |u|^2) / d on the grid v_j = -L + j h; +inf when rho <= 0, T <= 0 or
    sum |f| = 0."""
    f = _f64(f)
    d, N = f.ndim, f.shape[0]
    h = 2.0 * L / N
    axes = np.meshgrid(*([-L + h * np.arange(N)] * d), indexing="ij")
    rho = h ** d * f.sum()
    if not rho > 0.0:
        return float("inf")
    u = [h ** d * (f * v).sum() / rho for v in axes]
    T = (h ** d * (f * sum(v * v for v in axes)).sum() / rho - sum(x * x for x in u)) / d
    if not T > 0.0 or not np.isfinite(T):
        return float("inf")
    w2 = sum((v - x) ** 2 for v, x in zip(axes, u))
    M = rho * (2.0 * np.pi * T) ** (-0.5 * d) * np.exp(-w2 / (2.0 * T))
    den = np.abs(f).sum()
    return float(np.abs(f - M).sum() / den) if den > 0.0 else float("inf")


def rk2(f, L: float, Nbar: int, dt: float, n_steps: int, kernel: str = "unit",
        Ntilde: int | None = None) -> np.ndarray:
    """n_steps of the second-order total-variation-diminishing Runge-Kutta
    scheme that Section 4 uses for its runs, for df/dt = Q(f):
    f1 = f + dt Q(f), then f <- (f + f1 + dt Q(f1)) / 2."""
    f = _f64(f).copy()
    for _ in range(n_steps):
        f1 = f + dt * q(f, L, Nbar, kernel=kernel, Ntilde=Ntilde)["Q"]
        f = 0.5 * (f + (f1 + dt * q(f1, L, Nbar, kernel=kernel, Ntilde=Ntilde)["Q"]))
    return f


def jvp(f, df, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None) -> np.ndarray:
    f = _f64(f)
    df = _f64(df)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    out = np.zeros_like(f)
    rc = _load().oracle_jvp(d, N, Nt, m, KERNELS[kernel], h, _dp(f), _dp(df), _dp(out))
    if rc != 0:
        raise RuntimeError(f"oracle_jvp failed ({rc})")
    return out


def vjp(f, g, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None,
        with_scale: bool = False):
    """Transpose of the Jacobian applied to g (term-by-term scatter).  With
    ``with_scale`` also returns the scattered sum of absolute values."""
    f = _f64(f)
    g = _f64(g)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    out = np.zeros_like(f)
    sc = np.zeros_like(f)
    rc = _load().oracle_vjp_scale(d, N, Nt, m, KERNELS[kernel], h, _dp(f), _dp(g), _dp(out), _dp(sc))
    if rc != 0:
        raise RuntimeError(f"oracle_vjp failed ({rc})")
    return (out, sc) if with_scale else out


def jvp_points(f, df, L: float, Nbar: int, idx=None, kernel: str = "unit", Ntilde: int | None = None):
    """(dQ, scale) at flat indices ``idx`` (all points when None); scale is the
    sum of absolute values of the four products of every term."""
    f = _f64(f)
    df = _f64(df)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    if idx is None:
        n, ip = f.size, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n, ip = idx.size, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    out, sc = np.zeros(n), np.zeros(n)
    rc = _load().oracle_jvp_points(d, N, Nt, m, KERNELS[kernel], h, _dp(f), _dp(df), ip, n, _dp(out), _dp(sc))
    if rc != 0:
        raise RuntimeError(f"oracle_jvp_points failed ({rc})")
    if idx is None:
        out, sc = out.reshape(f.shape), sc.reshape(f.shape)
    return out, sc


def vjp_points(f, g, L: float, Nbar: int, idx, kernel: str = "unit", Ntilde: int | None = None):
    """(grad, scale) at flat indices ``idx``, summed as a gather over the
    terms in which each selected f_p appears."""
    f = _f64(f)
    g = _f64(g)
    d, N, Nt, m, h = _params(f, L, Nbar, Ntilde)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out, sc = np.zeros(idx.size), np.zeros(idx.size)
    rc = _load().oracle_vjp_points(d, N, Nt, m, KERNELS[kernel], h, _dp(f), _dp(g),
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), idx.size, _dp(out), _dp(sc))
    if rc != 0:
        raise RuntimeError(f"oracle_vjp_points failed ({rc})")
    return out, sc


def _weight(k, kernel: str, h: float, d: int) -> float:
    """a(k) of the decoupled weights after eq. (decoup): 1 (unit kernel) or
    h^{2d-1} |k| / gcd(k) (Heintz-Panferov weights, b(l) = 1)."""
    if kernel == "unit":
        return 1.0
    g = 0
    for x in k:
        g = np.gcd(g, abs(int(x)))
    return h ** (2 * d - 1) * float(np.sqrt(np.dot(k, k))) / g


def spectral_beta(d: int, N: int, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None) -> np.ndarray:
    """beta~(K, L) = beta(K, L) - beta(L, L) for K, L in Z_N^d (flat
    row-major indices), shape (N^d, N^d), real.

    beta(K, L) = sum_{k, l} Gamma(k) e_K(k) e_L(l) over the pairs of eq.
    (betaKL): k, l in [-Ntilde, Ntilde]^d minus 0 with k . l = 0 and the line
    of k in A_m (eq. (decDVM)), e_K(k) = exp(2 pi i K . k / N).  Summed pair
    by pair (grouped by k), without the line decomposition."""
    Nt = default_ntilde(N) if Ntilde is None else int(Ntilde)
    m = min(int(Nbar), Nt)
    h = 2.0 * L / N
    rng = np.arange(-Nt, Nt + 1)
    box = np.array(np.meshgrid(*([rng] * d), indexing="ij")).reshape(d, -1).T
    box = box[np.any(box != 0, axis=1)]
    modes = np.array(np.meshgrid(*([np.arange(N)] * d), indexing="ij")).reshape(d, -1).T
    ks, ws, S = [], [], []
    for k in box:
        g = 0
        for x in k:
            g = np.gcd(g, abs(int(x)))
        if np.max(np.abs(k // g)) > m:
            continue  # the line of k is not in A_m
        ls = box[box @ k == 0]
        if ls.size == 0:
            continue
        ks.append(k)
        ws.append(_weight(k, kernel, h, d))
        S.append(np.exp(2j * np.pi * (modes @ ls.T) / N).sum(axis=1))  # sum_l e_L(l)
    Ek = np.exp(2j * np.pi * (modes @ np.array(ks).T) / N)  # (N^d, #k)
    beta = (Ek * np.array(ws)) @ np.array(S)  # (N^d, N^d)
    if np.max(np.abs(beta.imag)) > 1e-9 * max(1.0, np.max(np.abs(beta.real))):
        raise RuntimeError("beta is not real: the term set is not symmetric")
    beta = beta.real
    return beta - np.diag(beta)[None, :]


def q_spectral(f, L: float, Nbar: int, kernel: str = "unit", Ntilde: int | None = None,
               beta: np.ndarray | None = None) -> np.ndarray:
    """Q through eq. (sysDiff): Qhat_I = sum_{K + L = I} beta~(K, L) fhat_K
    fhat_L with fhat_I = N^{-d} sum_i f_i e_{-I}(i), then Q_i = sum_I
    Qhat_I e_I(i)."""
    f = _f64(f)
    d, N = f.ndim, f.shape[0]
    if beta is None:
        beta = spectral_beta(d, N, L, Nbar, kernel, Ntilde)
    M = N ** d
    modes = np.array(np.meshgrid(*([np.arange(N)] * d), indexing="ij")).reshape(d, -1).T
    fh = np.fft.fftn(f).ravel() / M
    Qh = np.zeros(M, dtype=complex)
    for I in range(M):
        Lm = (modes[I][None, :] - modes) % N  # L = I - K for every K
        Li = np.ravel_multi_index(Lm.T, (N,) * d)
        Qh[I] = np.sum(beta[np.arange(M), Li] * fh * fh[Li])
    Q = np.fft.ifftn(Qh.reshape((N,) * d)) * M
    return Q.real


def moments(Q, L: float) -> np.ndarray:
    """h^d sum Q phi for phi = 1, v_0..v_{d-1}, |v|^2 (d + 2 values)."""
    Q = _f64(Q)
    d = Q.ndim
    N = Q.shape[0]
    out = np.zeros(d + 2)
    rc = _load().oracle_moments(d, N, float(L), _dp(Q), _dp(out))
    if rc != 0:
        raise RuntimeError(f"oracle_moments failed ({rc})")
    return out


def rel_linf(Q, Qref, scale) -> float:
    """max_i |Q_i - Qref_i| / max_i scale_i (error relative to the largest
    sum of absolute terms, so that near-equilibrium data with Q ~ 0 stay
    well posed)."""
    Q = np.asarray(Q, dtype=np.float64)
    Qref = np.asarray(Qref, dtype=np.float64)
    s = float(np.max(np.abs(scale)))
    if s == 0.0:
        return float(np.max(np.abs(Q - Qref)))
    return float(np.max(np.abs(Q - Qref)) / s)
