"""Pins for the oracle's collision operator (CPU, no GPU).

Each test ties the oracle to something other than itself:

* the Fourier-side form of the method, eq. (sysDiff) with the kernel modes
  beta of eq. (betaKL) replaced by the direction decomposition of eq.
  (decDVM), evaluated with numpy's FFT on tiny grids;
* the general DVM form eq. (TypicalDVM)/(Gammaijkl) (momentum and energy
  indicators instead of orthogonality), brute force on tiny grids;
* closed forms: Q(const) = 0, Q(delta) = 0, two deltas (discrete Thales
  circle), Q(Maxwellian) = 0 away from the periodic boundary;
* invariants: mass (Proposition 3.2), momentum and energy without aliasing
  (item 4 after eq. (weakpe)), H-theorem sign, translation and
  hyperoctahedral equivariance, parity (item 2 after eq. (weakpe));
* the derivative: Q is quadratic, so Q(f+d) - Q(f) - Q(d) is exactly the
  JVP, and <g, J d> = <J^T g, d>;
* moments of a Gaussian in closed form.
"""
import itertools
from math import gcd

import numpy as np
import pytest

import oracle
import synth


# ----------------------------------------------------------------- helpers

def box(d, R):
    return [np.array(v) for v in itertools.product(range(-R, R + 1), repeat=d) if any(v)]


def prim(v):
    g = 0
    for x in v:
        g = gcd(g, abs(int(x)))
    return np.array(v) // g, g


def a_weight(k, kernel, h, d):
    if kernel == "unit":
        return 1.0
    e, g = prim(k)
    return h ** (2 * d - 1) * float(np.linalg.norm(k)) / g


def directions(d, m):
    out = []
    for v in itertools.product(range(-m, m + 1), repeat=d):
        if not any(v):
            continue
        e, g = prim(v)
        if g != 1:
            continue
        first = next(x for x in v if x != 0)
        if first > 0:
            out.append(np.array(v))
    return out


def fourier_side(f, L, Nbar, kernel, Ntilde):
    """eq. (sysDiff): dhat_I = sum_{K+L=I} (beta(K,L) - beta(L,L)) f~_K f~_L
    with beta(K,L) = sum_e alpha_e(K) alpha'_e(L) (eq. (decDVM)),
    alpha_e(K) = sum_{k in eZ, 0<|k|<=Nt} a(k) e_K(k),
    alpha'_e(L) = sum_{l in e^perp, 0<|l|<=Nt} e_L(l),  e_K(k) = exp(2 pi i K.k / N)."""
    d = f.ndim
    N = f.shape[0]
    h = 2.0 * L / N
    m = min(Nbar, Ntilde)
    modes = np.array(list(itertools.product(range(N), repeat=d)))  # flat K order = row-major
    M = modes.shape[0]
    beta = np.zeros((M, M), dtype=complex)
    for e in directions(d, m):
        J = Ntilde // int(np.max(np.abs(e)))
        ks = [j * e for j in range(-J, J + 1) if j != 0]
        ls = [l for l in box(d, Ntilde) if int(np.dot(l, e)) == 0]
        alpha = sum(a_weight(k, kernel, h, d) * np.exp(2j * np.pi * modes @ k / N) for k in ks)
        alphap = sum(np.exp(2j * np.pi * modes @ l / N) for l in ls)
        beta += np.outer(alpha, alphap)
    ft = np.fft.fftn(f).ravel() / M
    # index of I - K for all (I, K)
    diff = (modes[:, None, :] - modes[None, :, :]) % N
    flat = np.zeros(diff.shape[:2], dtype=np.int64)
    for a in range(d):
        flat = flat * N + diff[..., a]
    Kidx = np.broadcast_to(np.arange(M)[None, :], (M, M))
    bt = beta[Kidx, flat] - beta[flat, flat]
    dhat = np.sum(bt * ft[Kidx] * ft[flat], axis=1)
    D = np.fft.ifftn(dhat.reshape((N,) * d)) * M
    assert np.max(np.abs(D.imag)) < 1e-10 * max(1.0, np.max(np.abs(D.real)))
    return D.real


def general_dvm(f, L, Nbar, kernel, Ntilde):
    """eq. (TypicalDVM): D_i = sum_{j,k',l'} Gamma_{ij}^{k'l'} [f_k' f_l' - f_i f_j]
    with the indicators 1(i+j-k'-l') 1(|i|^2+|j|^2-|k'|^2-|l'|^2) of eq.
    (Gammaijkl), post-collision velocities truncated to |k'-i|, |l'-i| <= Nt,
    the line of k'-i restricted to |e|_inf <= m, f read periodically."""
    d = f.ndim
    N = f.shape[0]
    h = 2.0 * L / N
    m = min(Nbar, Ntilde)
    B = box(d, Ntilde)
    out = np.zeros_like(f)
    for i in itertools.product(range(N), repeat=d):
        iv = np.array(i)
        acc = 0.0
        for k in B:
            e, _ = prim(k)
            if np.max(np.abs(e)) > m:
                continue
            w = a_weight(k, kernel, h, d)
            kp = iv + k
            for l in B:
                lp = iv + l
                j = kp + lp - iv
                if int(iv @ iv + j @ j - kp @ kp - lp @ lp) != 0:
                    continue
                acc += w * (f[tuple(kp % N)] * f[tuple(lp % N)] - f[i] * f[tuple(j % N)])
        out[i] = acc
    return out


def rng_f(shape, seed):
    return np.random.default_rng(seed).uniform(0.1, 1.0, size=shape)


# ------------------------------------------------------ independent forms

@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", [
    (2, 9, 3, 1, "unit"), (2, 9, 3, 2, "hp"), (2, 9, 3, 3, "unit"), (2, 8, 3, 2, "hp"),
    (3, 6, 2, 1, "hp"), (3, 6, 2, 2, "unit"),
])
def test_matches_fourier_side_decomposition(d, N, Nt, Nbar, kernel):
    f = rng_f((N,) * d, seed=11 + N + Nbar)
    L = 3.0
    ref = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    D = fourier_side(f, L, Nbar, kernel, Nt)
    assert oracle.rel_linf(ref["Q"], D, ref["scale"]) < 1e-12


@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", [(2, 7, 2, 2, "hp"), (2, 8, 3, 1, "unit"), (3, 5, 1, 1, "hp")])
def test_matches_general_dvm_form(d, N, Nt, Nbar, kernel):
    f = rng_f((N,) * d, seed=5 + N)
    L = 2.5
    ref = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    D = general_dvm(f, L, Nbar, kernel, Nt)
    assert oracle.rel_linf(ref["Q"], D, ref["scale"]) < 1e-13


# ---------------------------------------------------------- closed forms

@pytest.mark.parametrize("d,N,Nbar", [(2, 16, 3), (2, 20, 2), (3, 10, 2)])
def test_constant_and_single_delta_give_zero_exactly(d, N, Nbar):
    c = np.full((N,) * d, 0.37)
    for kernel in ("unit", "hp"):
        assert np.all(oracle.q(c, 4.0, Nbar, kernel=kernel)["Q"] == 0.0)
    delta = np.zeros((N,) * d)
    delta[(3,) * d] = 2.0
    assert np.all(oracle.q(delta, 4.0, Nbar, kernel="hp")["Q"] == 0.0)


def _rep(x, N):
    """Representative of x mod N in [-(N-1)//2, N//2]."""
    r = x % N
    return np.where(r > N // 2, r - N, r)


@pytest.mark.parametrize("d,N,Nt,Nbar,a,b", [
    (2, 16, 3, 3, (5, 5), (7, 6)), (2, 16, 3, 1, (5, 5), (7, 7)), (2, 18, 4, 2, (2, 3), (5, 1)),
    (3, 10, 2, 2, (4, 4, 4), (5, 6, 4)), (3, 10, 2, 1, (1, 2, 3), (3, 2, 3)),
])
def test_two_deltas_thales_circle(d, N, Nt, Nbar, a, b):
    """f = delta_a + delta_b, unit kernel.  Away from a and b, Q_p counts the
    ways p sees a and b at orthogonal displacements (one for each of a-p and
    b-p whose line is admissible); Q_a = -#{(k,l) in S: k+l = b-a}, same for
    b (the discrete Thales circle over the segment ab)."""
    assert 2 * Nt < N
    m = min(Nbar, Nt)
    f = np.zeros((N,) * d)
    f[a] = 1.0
    f[b] = 1.0
    Q = oracle.q(f, 4.0, Nbar, kernel="unit", Ntilde=Nt)["Q"]
    A, Bv = np.array(a), np.array(b)

    def admissible(k):
        if not np.any(k) or np.max(np.abs(k)) > Nt:
            return False
        e, _ = prim(k)
        return np.max(np.abs(e)) <= m

    expect = np.zeros_like(f)
    for p in itertools.product(range(N), repeat=d):
        P = np.array(p)
        if p in (a, b):
            continue
        ka, kb = _rep(A - P, N), _rep(Bv - P, N)
        if not (np.any(ka) and np.any(kb)) or max(np.max(np.abs(ka)), np.max(np.abs(kb))) > Nt:
            continue
        if int(ka @ kb) != 0:
            continue
        expect[p] = float(admissible(ka)) + float(admissible(kb))
    for src, dst in ((A, Bv), (Bv, A)):
        tgt = _rep(dst - src, N)
        cnt = 0
        for k in box(d, Nt):
            if not admissible(k):
                continue
            l = tgt - k
            if np.any(l) and np.max(np.abs(l)) <= Nt and int(k @ l) == 0:
                cnt += 1
        expect[tuple(src)] = -cnt
    assert np.array_equal(Q, expect)


def test_maxwellian_is_equilibrium_in_the_interior():
    for d, N, L in ((2, 32, 8.0), (3, 16, 6.0)):
        M = synth.maxwellian(d, N, L, 1.0, (0.3,) * d, 1.2)
        # a generic exp(a + b.v + c|v|^2) on a wider box as well
        for kernel in ("unit", "hp"):
            r = oracle.q(M, L, 8, kernel=kernel)
            Nt = oracle.default_ntilde(N)
            lim = N // 2 - 1 - 2 * Nt
            sl = tuple(slice(N // 2 - lim, N // 2 + lim + 1) for _ in range(d))
            assert np.max(np.abs(r["Q"][sl]) / r["scale"][sl]) < 1e-13
            # everywhere: only aliasing terms, tiny for this width
            assert oracle.rel_linf(r["Q"], 0 * r["Q"], r["scale"]) < 1e-6


# ----------------------------------------------------------- invariants

@pytest.mark.parametrize("d,N,Nbar,kernel", [(2, 16, 2, "unit"), (2, 24, 3, "hp"), (3, 10, 1, "hp"), (3, 12, 2, "unit")])
def test_mass_conserved_for_any_data(d, N, Nbar, kernel):
    f = rng_f((N,) * d, seed=3)
    r = oracle.q(f, 5.0, Nbar, kernel=kernel)
    assert abs(r["Q"].sum()) <= 1e-14 * r["scale"].sum()


@pytest.mark.parametrize("d,N,Nbar,kernel", [(2, 24, 3, "hp"), (2, 32, 2, "unit"), (3, 16, 2, "hp")])
def test_momentum_energy_conserved_without_aliasing(d, N, Nbar, kernel):
    Nt = oracle.default_ntilde(N)
    S = N // 2 - 1 - Nt
    f = synth.compact_support(d, N, S, seed=4)
    L = 5.0
    r = oracle.q(f, L, Nbar, kernel=kernel)
    vs = synth.grid(d, N, L)
    phis = [np.ones_like(f)] + vs + [sum(v * v for v in vs)]
    for phi in phis:
        num = abs(np.sum(r["Q"] * phi))
        den = np.sum(r["scale"] * np.abs(phi))
        assert num <= 1e-13 * den
    # and with aliasing momentum/energy are *not* conserved in general
    g = rng_f((N,) * d, seed=9)
    rg = oracle.q(g, L, Nbar, kernel=kernel)
    e2 = sum(v * v for v in vs)
    assert abs(np.sum(rg["Q"] * e2)) > 1e-8 * np.sum(rg["scale"] * e2)


@pytest.mark.parametrize("d,N,Nbar", [(2, 16, 3), (3, 10, 2)])
def test_h_theorem_sign(d, N, Nbar):
    for seed in range(4):
        f = rng_f((N,) * d, seed=seed)
        Q = oracle.q(f, 4.0, Nbar, kernel="hp")["Q"]
        assert np.sum(Q * np.log(f)) <= 1e-15


@pytest.mark.parametrize("d,N,Nbar", [(2, 14, 2), (3, 9, 2)])
def test_equivariance_translation_and_hyperoctahedral(d, N, Nbar):
    f = rng_f((N,) * d, seed=21)
    for kernel in ("unit", "hp"):
        Q = oracle.q(f, 4.0, Nbar, kernel=kernel)["Q"]
        sh = tuple(range(1, d + 1))
        Qs = oracle.q(np.roll(f, sh, axis=tuple(range(d))), 4.0, Nbar, kernel=kernel)["Q"]
        assert np.allclose(Qs, np.roll(Q, sh, axis=tuple(range(d))), rtol=0, atol=1e-14)
        for ax in range(d):
            Qf = oracle.q(np.flip(f, axis=ax).copy(), 4.0, Nbar, kernel=kernel)["Q"]
            assert np.allclose(Qf, np.flip(Q, axis=ax), rtol=0, atol=1e-14)
        perm = tuple(reversed(range(d)))
        Qt = oracle.q(np.transpose(f, perm).copy(), 4.0, Nbar, kernel=kernel)["Q"]
        assert np.allclose(Qt, np.transpose(Q, perm), rtol=0, atol=1e-14)


def test_gain_nonnegative_and_parity():
    N = 16
    f = rng_f((N, N), seed=2)
    r = oracle.q(f, 4.0, 3)
    assert np.all(r["gain"] >= 0) and np.all(r["loss"] >= 0)
    assert np.allclose(r["gain"] - r["loss"], r["Q"], atol=1e-15)
    # even f (f(-v) = f(v) on the torus) gives even Q and zero momentum
    idx = (-np.arange(N)) % N
    fe = f + f[np.ix_(idx, idx)]
    Qe = oracle.q(fe, 4.0, 3)["Q"]
    assert np.allclose(Qe, Qe[np.ix_(idx, idx)], atol=1e-14)


def test_restricted_equals_full_at_nbar_ntilde_and_differs_below():
    N = 24
    f = rng_f((N, N), seed=8)
    Nt = oracle.default_ntilde(N)
    full = oracle.q(f, 4.0, 100)["Q"]
    at = oracle.q(f, 4.0, Nt)["Q"]
    assert np.array_equal(full, at)
    below = oracle.q(f, 4.0, Nt - 2)["Q"]
    assert np.max(np.abs(below - full)) > 1e-6


def test_q_points_matches_full_evaluation():
    f = rng_f((3 * 4,) * 3, seed=1)
    r = oracle.q(f, 3.0, 2, kernel="hp")
    idx = np.array([0, 5, 77, 1000, 1727])
    rp = oracle.q_points(f, 3.0, 2, idx, kernel="hp")
    assert np.array_equal(rp["Q"], r["Q"].ravel()[idx])
    assert np.array_equal(rp["scale"], r["scale"].ravel()[idx])


# ----------------------------------------------------------- derivatives

@pytest.mark.parametrize("d,N,Nbar,kernel", [(2, 12, 2, "hp"), (3, 8, 1, "unit")])
def test_jvp_is_the_quadratic_polarisation(d, N, Nbar, kernel):
    f = rng_f((N,) * d, seed=31)
    dl = np.random.default_rng(32).standard_normal((N,) * d)
    L = 3.0
    J = oracle.jvp(f, dl, L, Nbar, kernel=kernel)
    rf = oracle.q(f + dl, L, Nbar, kernel=kernel)
    diff = rf["Q"] - oracle.q(f, L, Nbar, kernel=kernel)["Q"] - oracle.q(dl, L, Nbar, kernel=kernel)["Q"]
    assert oracle.rel_linf(J, diff, rf["scale"]) < 1e-13
    eps = 1e-3
    fd = (oracle.q(f + eps * dl, L, Nbar, kernel=kernel)["Q"] - oracle.q(f - eps * dl, L, Nbar, kernel=kernel)["Q"]) / (2 * eps)
    assert oracle.rel_linf(J, fd, rf["scale"]) < 1e-9


@pytest.mark.parametrize("d,N,Nbar,kernel", [(2, 12, 3, "hp"), (3, 8, 2, "unit")])
def test_vjp_is_the_transpose_of_jvp(d, N, Nbar, kernel):
    f = rng_f((N,) * d, seed=41)
    rs = np.random.default_rng(42)
    g = rs.standard_normal((N,) * d)
    L = 3.0
    G = oracle.vjp(f, g, L, Nbar, kernel=kernel)
    for _ in range(3):
        dl = rs.standard_normal((N,) * d)
        lhs = np.sum(g * oracle.jvp(f, dl, L, Nbar, kernel=kernel))
        rhs = np.sum(G * dl)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sum(np.abs(g)) * 1e-3)
    # explicit Jacobian column check at one point
    e = np.zeros_like(f)
    e[(1,) * d] = 1.0
    col = oracle.jvp(f, e, L, Nbar, kernel=kernel)
    assert abs(np.sum(g * col) - G[(1,) * d]) < 1e-12 * np.sum(np.abs(col) * np.abs(g)) + 1e-15


# ---------------------------------------------------------------- moments

def test_moments_of_gaussian_closed_form():
    for d, N, L in ((2, 64, 10.0), (3, 32, 9.0)):
        u = np.array([0.4, -0.3, 0.2][:d])
        T = 0.9
        M = synth.maxwellian(d, N, L, 1.3, u, T)
        m = oracle.moments(M, L)
        assert abs(m[0] - 1.3) < 1e-10
        assert np.allclose(m[1:1 + d], 1.3 * u, atol=1e-10)
        assert abs(m[d + 1] - 1.3 * (u @ u + d * T)) < 1e-9


@pytest.mark.parametrize("d,N,Nbar,kernel", [(2, 11, 2, "hp"), (3, 7, 1, "unit")])
def test_points_variants_match_full_arrays(d, N, Nbar, kernel):
    """jvp_points equals jvp; vjp_points (gather) equals vjp (scatter)."""
    rs = np.random.default_rng(51)
    f = rs.uniform(0.1, 1.0, (N,) * d)
    g = rs.standard_normal((N,) * d)
    dl = rs.standard_normal((N,) * d)
    idx = np.array([0, 3, N ** d // 2, N ** d - 1])
    J = oracle.jvp(f, dl, 2.0, Nbar, kernel=kernel)
    Jp, Js = oracle.jvp_points(f, dl, 2.0, Nbar, idx, kernel=kernel)
    assert np.allclose(Jp, J.ravel()[idx], rtol=0, atol=1e-14 * np.max(Js))
    G, Gs = oracle.vjp(f, g, 2.0, Nbar, kernel=kernel, with_scale=True)
    Gp, Gps = oracle.vjp_points(f, g, 2.0, Nbar, idx, kernel=kernel)
    assert np.allclose(Gp, G.ravel()[idx], rtol=0, atol=1e-14 * np.max(Gs))
    assert np.allclose(Gps, Gs.ravel()[idx], rtol=1e-13)
    # the scales bound the values
    assert np.all(np.abs(G) <= Gs * (1 + 1e-12)) and np.all(np.abs(Jp) <= Js * (1 + 1e-12))
