"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
closed form the paper derives, a textbook special case, an exact invariant, or a
brute-force construction on a tiny grid.
"""
import numpy as np
import pytest

from paper_1804_01390_gb300 import workloads as wk


# ----------------------------------------------------------------------------------
# Thm 1.1 (eq:IntroSolution, eq:IntroDecayRate) and the Fourier-domain aux fields
# (eq:PhiDefinitionA, eq:PsiDefinitionA): the extended travelling wave is an exact
# eigenvector of the semi-discrete operator, A y = -i omega y, for ANY sigma >= 0.
# ----------------------------------------------------------------------------------

def _rho(s, k, omega, h):
    """One-cell decay rate, eq:IntroDecayRate."""
    return ((2 + 1j * s / omega * (1 - np.exp(-1j * k * h)))
            / (2 + 1j * s / omega * (1 - np.exp(1j * k * h))))


def _axis_fields(sig, k, omega, h):
    """1D factors R W, Phi-hat, Psi-hat on vertices 0..T-1 of one axis.

    R(i) = prod_{j<i} rho(sigma(j)) (eq:IntroSolution), and
    Phi(i) = (R(i+1)W(i+1) - R(i)W(i-1)) / (i omega h (2 + i sigma(i)/omega)),
    Psi(i) = (R(i)W(i+1) - R(i-1)W(i-1)) / (i omega h (2 + i sigma(i-1)/omega)),
    which is eq:PhiDefinitionA / eq:PsiDefinitionA with f restricted to the
    stretching path via Thm 3.1 (eq:DecayRate).
    """
    T = sig.shape[0]
    R = np.ones(T + 2, dtype=complex)   # R[j+1] = R(j) for j = -1..T
    R[0] = 1.0 / _rho(sig[T - 1], k, omega, h)
    for j in range(T):
        R[j + 2] = R[j + 1] * _rho(sig[j], k, omega, h)
    Rf = lambda j: R[j + 1]
    W = lambda j: np.exp(1j * k * h * j)
    i = np.arange(T)
    u = Rf(i) * W(i)
    sm1 = np.roll(sig, 1)
    phi = (Rf(i + 1) * W(i + 1) - Rf(i) * W(i - 1)) / (1j * omega * h * (2 + 1j * sig / omega))
    psi = (Rf(i) * W(i + 1) - Rf(i - 1) * W(i - 1)) / (1j * omega * h * (2 + 1j * sm1 / omega))
    return u, phi, psi


def _plane_wave_state(T, sigmas, ks, h):
    nd = len(T)
    omega = np.sqrt(sum(4 * np.sin(k * h / 2) ** 2 for k in ks)) / h
    omega = complex(omega)
    ax = [_axis_fields(s, k, omega, h) for s, k in zip(sigmas, ks)]
    shape = T[::-1]

    def outer(factors):
        out = np.ones(shape, dtype=complex)
        for a, f in enumerate(factors):
            sh = [1] * nd
            sh[nd - 1 - a] = T[a]
            out = out * f.reshape(sh)
        return out

    U = outer([ax[a][0] for a in range(nd)])
    fields = [U, -1j * omega * U]
    for a in range(nd):
        fa = [ax[b][0] for b in range(nd)]
        fa[a] = ax[a][1]
        fields.append(outer(fa))
        fa[a] = ax[a][2]
        fields.append(outer(fa))
    return omega, np.stack([f.reshape(-1) for f in fields])


def _check_eigen(orc, T, sigmas, ks, h=1.0, tol=1e-12):
    g = orc.Grid(T, h, sigmas)
    omega, y = _plane_wave_state(T, sigmas, ks, h)
    lam = -1j * omega
    Ar = orc.rhs(g, y.real)
    Ai = orc.rhs(g, y.imag)
    Ay = Ar + 1j * Ai
    # rows whose stencil does not cross the periodic wrap
    nd = len(T)
    idx = np.indices(T[::-1])
    ok = np.ones(T[::-1], dtype=bool)
    for a in range(nd):
        c = idx[nd - 1 - a]
        ok &= (c >= 1) & (c <= T[a] - 2)
    ok = ok.reshape(-1)
    scale = np.abs(y).max()
    err = 0.0
    for f in range(2 + 2 * nd):
        rows = ok.copy()
        if f >= 2:
            a = (f - 2) // 2
            sig = sigmas[a]
            coords = idx[nd - 1 - a].reshape(-1)
            active = sig[coords] != 0 if f % 2 == 0 else np.roll(sig, 1)[coords] != 0
            rows &= active
        err = max(err, np.abs(Ay[f, rows] - lam * y[f, rows]).max() / scale)
    assert err < tol, err
    return err


@pytest.mark.parametrize("kh", [0.3, 1.1, 2.3, 3.0])
def test_plane_wave_is_eigenvector_1d_random_sigma(orc, kh):
    rng = np.random.default_rng(10)
    T = 40
    sig = np.zeros(T)
    sig[18:] = rng.uniform(0, 2.0, size=T - 18)   # half-space layer, i.i.d. U[0, 2/h]
    _check_eigen(orc, (T,), [sig], [kh])


def test_plane_wave_is_eigenvector_2d_oblique(orc):
    rng = np.random.default_rng(11)
    T = (22, 19)
    sigs = []
    for t in T:
        s = np.zeros(t)
        s[t // 2:] = rng.uniform(0, 2.0, size=t - t // 2)
        sigs.append(s)
    _check_eigen(orc, T, sigs, [0.7, 2.1])


def test_evanescent_wave_is_eigenvector_2d(orc):
    # k_y complex with Im k < 0 (eq:KDomain) and real omega through eq:DiscreteDispersion
    h = 1.0
    kx = 0.4
    omega = 0.2
    s2 = (omega ** 2 * h ** 2 - 4 * np.sin(kx * h / 2) ** 2) / 4
    ky = 2 * np.arcsin(np.sqrt(complex(s2))) / h
    if ky.imag > 0:
        ky = np.conj(ky)
    assert ky.imag < 0
    rng = np.random.default_rng(12)
    T = (20, 18)
    sigs = [np.concatenate([np.zeros(t // 2), rng.uniform(0, 2, t - t // 2)]) for t in T]
    _check_eigen(orc, T, sigs, [kx, ky], tol=1e-11)


def test_plane_wave_is_eigenvector_3d(orc):
    rng = np.random.default_rng(13)
    T = (11, 10, 9)
    sigs = [np.concatenate([np.zeros(t // 2), rng.uniform(0, 2, t - t // 2)]) for t in T]
    _check_eigen(orc, T, sigs, [0.5, 1.7, 2.6])


def test_plane_wave_dx_not_one(orc):
    rng = np.random.default_rng(14)
    h = 1.0 / 80.0   # the paper's grid size in Fig. HalfSpaceGauss
    T = 30
    sig = np.concatenate([np.zeros(12), rng.uniform(0, 2.0 / h, T - 12)])
    _check_eigen(orc, (T,), [sig], [1.3 / h], h=h)


# ----------------------------------------------------------------------------------
# Thm 3.2: |rho| < 1 and |rho(k)| / |rho(-conj k)| < 1 for right-travelling waves;
# rho(0, k, omega) = 1; k = 0 and pi/h cases of App. A.  These pin the closed form
# used above (so that a wrong rho would not pass the eigenvector tests by accident).
# ----------------------------------------------------------------------------------

def test_decay_rate_properties():
    rng = np.random.default_rng(15)
    h = 1.0
    for _ in range(2000):
        s = rng.uniform(1e-3, 5.0)
        om = rng.uniform(0.05, 2.8) * (1 if rng.random() < 0.5 else -1)
        kr = rng.uniform(1e-3, np.pi - 1e-3) * np.sign(om)
        ki = -rng.uniform(0, 2.0)
        k = kr + 1j * ki
        r = _rho(s, k, om, h)
        assert abs(r) < 1
        assert abs(r) / abs(_rho(s, -np.conj(k), om, h)) < 1
    assert abs(_rho(0.0, 0.9, 0.7, h) - 1) == 0
    assert abs(_rho(1.3, 0.0, 0.7, h) - 1) < 1e-15          # App. A, case k = 0
    assert abs(_rho(1.3, np.pi, 0.7, h) - 1) < 1e-15        # case k = pi/h: f o L1 = -W = rho tau W


# ----------------------------------------------------------------------------------
# Classic RK4 on a single Fourier mode (sigma = 0): the mode evolves by the 2x2
# Taylor polynomial P(dt M), M = [[0,1],[-omega^2,0]], omega from eq:DiscreteDispersion,
# and the energy eq:Energy of the mode is multiplied by |R(i omega dt)|^2 per step.
# ----------------------------------------------------------------------------------

def _mode(T, m):
    idx = np.indices(T[::-1])
    th = np.zeros(T[::-1])
    for a in range(len(T)):
        th = th + 2 * np.pi * m[a] * idx[len(T) - 1 - a] / T[a]
    return np.cos(th).reshape(-1)


@pytest.mark.parametrize("T,m,dt,h", [((16, 12), (3, 2), 0.5, 1.0), ((9, 8, 10), (2, 3, 4), 0.4, 1.0),
                                      ((32,), (7,), 0.9, 1.0), ((16, 12), (3, 2), 0.3, 0.6)])
def test_rk4_single_mode_exact(orc, T, m, dt, h):
    g = orc.Grid(T, h, [np.zeros(t) for t in T])
    om2 = sum(4 * np.sin(np.pi * mm / t) ** 2 for mm, t in zip(m, T)) / h ** 2
    y = g.zeros_state()
    y[0] = _mode(T, m)
    n = 37
    yn, _ = orc.rk4(g, y, n, dt)
    M = np.array([[0, 1.0], [-om2, 0]])
    P = np.eye(2) + dt * M + (dt * M) @ (dt * M) / 2 + np.linalg.matrix_power(dt * M, 3) / 6 \
        + np.linalg.matrix_power(dt * M, 4) / 24
    uv = np.linalg.matrix_power(P, n) @ np.array([1.0, 0.0])
    assert np.abs(yn[0] - uv[0] * y[0]).max() < 1e-12
    assert np.abs(yn[1] - uv[1] * y[0]).max() < 1e-12
    # energy: mode energy n*omega^2/4 at V=0 (closed form of eq:Energy for a cosine mode)
    E0 = orc.energy(g, y)
    assert abs(E0 - g.n * om2 / 4) < 1e-10 * E0
    z = 1j * np.sqrt(om2) * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    En = orc.energy(g, yn)
    assert abs(En - E0 * abs(R) ** (2 * n)) < 1e-11 * E0


def test_wall_box_sine_mode_exact(orc):
    """With reflecting walls (every field zero at the vertices -1 and T_a) and no damping,
    products of sin(pi m_a (i_a + 1) / (T_a + 1)) are the eigenvectors of the discrete
    Laplacian with eigenvalue -sum_a 4 sin^2(pi m_a / (2 (T_a + 1))) / h^2, so one mode
    evolves by the 2 x 2 RK4 polynomial; a periodic seam at either end breaks this."""
    T, m, h, dt, n = (13, 9), (3, 2), 0.8, 0.35, 29
    g = orc.Grid(T, h, [np.zeros(t) for t in T], wall=True)
    idx = np.indices(T[::-1])
    u = np.ones(T[::-1])
    for a in range(2):
        u = u * np.sin(np.pi * m[a] * (idx[1 - a] + 1) / (T[a] + 1))
    om2 = sum(4 * np.sin(np.pi * mm / (2 * (t + 1))) ** 2 for mm, t in zip(m, T)) / h ** 2
    y = g.zeros_state()
    y[0] = u.reshape(-1)
    yn, _ = orc.rk4(g, y, n, dt)
    M = np.array([[0, 1.0], [-om2, 0]])
    P = np.eye(2) + dt * M + (dt * M) @ (dt * M) / 2 + np.linalg.matrix_power(dt * M, 3) / 6 \
        + np.linalg.matrix_power(dt * M, 4) / 24
    uv = np.linalg.matrix_power(P, n) @ np.array([1.0, 0.0])
    assert np.abs(yn[0] - uv[0] * y[0]).max() < 1e-12
    assert np.abs(yn[1] - uv[1] * y[0]).max() < 1e-12


def test_energy_is_additive_over_windows(orc):
    """eq:Energy is a sum of per-vertex terms: the windows [lo, k] and [k+1, hi] along any
    axis add up to [lo, hi] (inclusive bounds, each vertex counted once)."""
    rng = np.random.default_rng(28)
    T = (11, 9, 7)
    g = orc.Grid(T, 0.7, [np.zeros(t) for t in T])
    y = g.zeros_state()
    y[0] = rng.normal(size=g.n)
    y[1] = rng.normal(size=g.n)
    lo, hi = [1, 2, 0], [9, 7, 5]
    whole = orc.energy(g, y, lo, hi)
    for a in range(3):
        k = (lo[a] + hi[a]) // 2
        h1, l2 = list(hi), list(lo)
        h1[a], l2[a] = k, k + 1
        parts = orc.energy(g, y, lo, h1) + orc.energy(g, y, l2, hi)
        assert abs(parts - whole) < 1e-12 * whole
    assert orc.energy(g, y, [0, 0, 0], [t - 1 for t in T]) > whole


def test_energy_of_a_point_at_the_window_corners(orc):
    """eq:Energy by hand for U = u at one vertex p: the forward difference (tau_a U - U)/h
    equals -u/h at p and +u/h at p - e_a, so each axis gives u^2/h^2 when both vertices
    lie in the window (p at its upper corner) and u^2/(2h^2) when p - e_a lies outside it
    (p at its lower corner)."""
    T, h, u = (9, 8, 7), 0.6, 1.7
    g = orc.Grid(T, h, [np.zeros(t) for t in T])
    lo, hi = (2, 1, 3), (6, 5, 5)
    for p, per_axis in ((hi, u * u / h ** 2), (lo, u * u / (2 * h ** 2))):
        y = g.zeros_state()
        y[0, g.flat(p)] = u
        assert abs(orc.energy(g, y, lo, hi) - 3 * per_axis) < 1e-13 * per_axis


def test_norms_over_a_window(orc):
    """max |U|, the L2 norm and the L2 distance to a reference over an inclusive window,
    against numpy on the same slice."""
    rng = np.random.default_rng(29)
    T = (13, 10)
    g = orc.Grid(T, 1.0, [np.zeros(t) for t in T])
    U = rng.normal(size=T[::-1])
    ref = rng.normal(size=T[::-1])
    lo, hi = (2, 3), (11, 8)
    win = (slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
    mx, l2, d2 = orc.norms(g, U, ref, lo, hi)
    assert mx == np.abs(U[win]).max()
    assert abs(l2 - np.linalg.norm(U[win])) < 1e-13 * l2
    assert abs(d2 - np.linalg.norm(U[win] - ref[win])) < 1e-13 * d2
    assert orc.norms(g, U, None, lo, hi)[2] == 0.0


def test_energy_closed_form_velocity_mode(orc):
    T = (12, 10)
    g = orc.Grid(T, 0.5, [np.zeros(t) for t in T])
    y = g.zeros_state()
    y[1] = _mode(T, (1, 4))
    assert abs(orc.energy(g, y) - g.n / 4) < 1e-12 * g.n


# ----------------------------------------------------------------------------------
# RK4 with a time-dependent forcing: a spatially uniform source has LU = 0, so the
# constant mode solves U'' = a g(t) and RK4 reduces to Simpson's rule for V and
# U_1 = dt^2/6 (g(t) + 2 g(t+dt/2)) from rest (stage times 0, dt/2, dt/2, dt).
# ----------------------------------------------------------------------------------

def test_source_stage_times_simpson(orc):
    T = (6, 5)
    g = orc.Grid(T, 1.0, [np.zeros(t) for t in T])
    f, t0, dt = 0.1, 15.0, 0.5
    amp = 0.7
    src = {"idx": np.arange(g.n), "amp": np.full(g.n, amp), "f_peak": f, "t_delay": t0}
    y = g.zeros_state()
    step0 = 23
    y1, _ = orc.rk4(g, y, 1, dt, step0=step0, sources=src)
    t = step0 * dt

    def ric(tt):   # Ricker wavelet, written from its definition
        a = (np.pi * f * (tt - t0)) ** 2
        return (1 - 2 * a) * np.exp(-a)

    g1, g2, g4 = ric(t), ric(t + dt / 2), ric(t + dt)
    assert np.abs(y1[1] - amp * dt / 6 * (g1 + 4 * g2 + g4)).max() < 1e-15
    assert np.abs(y1[0] - amp * dt ** 2 / 6 * (g1 + 2 * g2)).max() < 1e-15


def test_ricker_definition(orc):
    f, t0 = 0.1, 15.0
    assert orc.ricker(t0, f, t0) == 1.0
    tz = t0 + 1 / (np.pi * f * np.sqrt(2))
    assert abs(orc.ricker(tz, f, t0)) < 1e-15
    ts = np.linspace(t0 - 60, t0 + 60, 24001)
    vals = np.array([orc.ricker(t, f, t0) for t in ts])
    assert abs(np.trapezoid(vals, ts)) < 1e-9     # zero mean wavelet


# ----------------------------------------------------------------------------------
# One RK4 step equals the degree-4 Taylor polynomial of dt*A for a linear autonomous
# system (brute force with the dense matrix of A on a tiny grid with a layer).
# ----------------------------------------------------------------------------------

def _dense_A(orc, g):
    N = g.nfields * g.n
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = orc.rhs(g, e).reshape(-1)
    return A


def _random_state(g, rng):
    y = rng.normal(size=(g.nfields, g.n))
    nd = g.ndim
    idx = np.indices(g.T[::-1])
    for a in range(nd):
        c = idx[nd - 1 - a].reshape(-1)
        s = g.sigmas[a]
        y[2 + 2 * a, s[c] == 0] = 0.0
        y[3 + 2 * a, np.roll(s, 1)[c] == 0] = 0.0
    return y


def test_rk4_step_equals_taylor_polynomial(orc):
    rng = np.random.default_rng(16)
    sx = orc.sigma_profile(3, 2, orc.KIND_POWER, 2.0, 2.0)
    sy = orc.sigma_profile(2, 2, orc.KIND_CONSTANT, 1.5)
    g = orc.Grid((7, 6), 1.0, [sx, sy])
    A = _dense_A(orc, g)
    dt = 0.45
    P = np.eye(A.shape[0])
    term = np.eye(A.shape[0])
    for k in range(1, 5):
        term = term @ (dt * A) / k
        P = P + term
    y = _random_state(g, rng)
    y1, _ = orc.rk4(g, y, 1, dt)
    assert np.abs(y1.reshape(-1) - P @ y.reshape(-1)).max() < 1e-13


def test_dense_spectral_radius_stable(orc):
    # Sec. 1.1.5: empirical stability, constant and random sigma, periodic truncation
    rng = np.random.default_rng(17)
    for sig in (orc.sigma_profile(6, 4, orc.KIND_CONSTANT, 2.0),
                orc.sigma_profile(6, 4, orc.KIND_RANDOM, 2.0, draws=rng.random(14))):
        g = orc.Grid((14,), 1.0, [sig])
        A = _dense_A(orc, g)
        for dt in (0.5, 1.0):
            P = np.eye(A.shape[0])
            term = np.eye(A.shape[0])
            for k in range(1, 5):
                term = term @ (dt * A) / k
                P = P + term
            rad = np.abs(np.linalg.eigvals(P)).max()
            assert rad <= 1 + 1e-6, rad


# ----------------------------------------------------------------------------------
# Damping profile and layout tables (conventions: edge-centred sigma, depth d_e).
# ----------------------------------------------------------------------------------

def test_sigma_profile_shapes(orc):
    N, w = 20, 6
    s = orc.sigma_profile(N, w, orc.KIND_POWER, 2.0, 2.0)
    T = N + 2 * w
    assert s.shape == (T,)
    a, b = w, w + N - 1
    assert np.all(s[a - 1:b + 1] == 0)            # physical edges and both interface edges
    assert np.count_nonzero(s) == 2 * w - 1
    assert s[T - 1] == 2.0                        # wrap edge: depth w
    assert s[b + 1] == 2.0 / w ** 2               # first layer edge: depth 1
    assert s[a - 2] == 2.0 / w ** 2
    m = np.array([s[(T - 2 - e) % T] for e in range(T)])   # mirror of edges
    assert np.array_equal(m, s)
    c = orc.sigma_profile(N, w, orc.KIND_CONSTANT, 1.0)
    assert np.count_nonzero(c) == 2 * w - 1 and c.max() == 1.0
    z = orc.sigma_profile(N, 0, orc.KIND_POWER, 2.0, 2.0)
    assert z.shape == (N,) and not z.any()


def test_interior_run_is_where_layer_terms_vanish(orc):
    """Interior vertices: one RK4 step of Eq. 3 equals the sigma=0 step exactly."""
    rng = np.random.default_rng(18)
    N, w = 14, 5
    for kind in (orc.KIND_POWER, orc.KIND_CONSTANT, orc.KIND_RANDOM):
        s = orc.sigma_profile(N, w, kind, 2.0, 2.0, draws=rng.random(N + 2 * w))
        T = N + 2 * w
        pa, qa, it = orc.layout_axis(s, w + N // 2)
        assert np.array_equal(pa, (s != 0).astype(np.uint8))
        assert np.array_equal(qa, (np.roll(s, 1) != 0).astype(np.uint8))
        run = np.flatnonzero(it)
        assert run.min() == w + 1 and run.max() == w + N - 2 and len(run) == N - 2
        g = orc.Grid((T,), 1.0, [s])
        g0 = orc.Grid((T,), 1.0, [np.zeros(T)])
        y = _random_state(g, rng)
        y0 = y.copy()
        y0[2:] = 0.0
        y1, _ = orc.rk4(g, y, 1, 0.5)
        y01, _ = orc.rk4(g0, y0, 1, 0.5)
        same = (y1[0] == y01[0]) & (y1[1] == y01[1])
        assert np.all(same[it == 1])
        assert not same[w].all() or not same[w + N - 1].all()   # just outside the run


# ----------------------------------------------------------------------------------
# Mirror symmetry: i -> T-1-i with Phi(i) -> -Psi(m(i)), Psi(i) -> -Phi(m(i)) maps
# solutions to solutions (the layer on the left is the mirror image of the right).
# ----------------------------------------------------------------------------------

def _mirror(g, y):
    nd = g.ndim
    out = np.empty_like(y)
    for f in range(g.nfields):
        out[f] = g.field(y, f)[tuple(slice(None, None, -1) for _ in range(nd))].reshape(-1)
    # axis-wise swap and sign for the aux fields of every axis: a full mirror flips all axes
    for a in range(nd):
        phi, psi = out[2 + 2 * a].copy(), out[3 + 2 * a].copy()
        out[2 + 2 * a] = -psi
        out[3 + 2 * a] = -phi
    return out


@pytest.mark.parametrize("T_N_w", [((12,), 4), ((10, 9), 3)])
def test_mirror_symmetry(orc, T_N_w):
    Ns, w = T_N_w
    rng = np.random.default_rng(19)
    sig = [orc.sigma_profile(n, w, orc.KIND_POWER, 2.0, 2.0) for n in Ns]
    g = orc.Grid(tuple(n + 2 * w for n in Ns), 1.0, sig)
    y = _random_state(g, rng)
    a, _ = orc.rk4(g, y, 5, 0.5)
    b, _ = orc.rk4(g, _mirror(g, y), 5, 0.5)
    assert np.abs(_mirror(g, a) - b).max() < 1e-12 * np.abs(a).max()


# ----------------------------------------------------------------------------------
# Reflectionless interface (Sec. 1.1.3, Fig. HalfSpaceGauss / HalfSpaceRand): before any
# residual wave can return, the PML-truncated solution equals the free-space solution on
# a box whose boundary is never reached, to machine zero, for constant and random sigma.
# ----------------------------------------------------------------------------------

def _truncated_vs_big(orc, N, w, sig_fn, steps, M, u0_small, dt=0.5):
    sigs = [sig_fn() for _ in range(2)]
    T = (N + 2 * w, N + 2 * w)
    g = orc.Grid(T, 1.0, sigs)
    y = g.zeros_state()
    y[0] = u0_small.reshape(-1)
    yn, _ = orc.rk4(g, y, steps, dt)
    gb = orc.Grid((M, M), 1.0, [np.zeros(M), np.zeros(M)])
    off = (M - N) // 2
    ub = np.zeros((M, M))
    ub[off:off + N, off:off + N] = u0_small[w:w + N, w:w + N]
    yb = gb.zeros_state()
    yb[0] = ub.reshape(-1)
    ybn, _ = orc.rk4(gb, yb, steps, dt)
    a = g.field(yn, 0)[w:w + N, w:w + N]
    b = gb.field(ybn, 0)[off:off + N, off:off + N]
    return np.abs(a - b).max(), np.abs(b).max()


def test_reflectionless_gauss_constant_sigma(orc):
    # w = 32: the path left layer -> periodic wrap -> right layer is 64 cells long, so no
    # residual wave re-enters within 40 steps (at w = 16 one arrives at the far interface
    # at ~2.5e-13 by step 40: that is Sec. 1.1.4's residual wave, not a reflection)
    N, w = 32, 32
    wl = wk.Workload("t", 2, (N, N), w, gaussians=[wk.Gaussian((w + 7.0, w + 15.5), 3.0, 2.0)])
    u0 = wk.initial_field(wl)
    err, ref = _truncated_vs_big(orc, N, w, lambda: orc.sigma_profile(N, w, orc.KIND_CONSTANT, 2.0),
                                 40, 160, u0)
    assert ref > 1e-2
    assert err < 1e-14, err


def test_reflectionless_noise_random_sigma(orc):
    N, w = 32, 32
    rng = np.random.default_rng(20)
    u0 = wk.white_noise_disk((N + 2 * w,) * 2, (w + 8.0, w + 16.0), 6.0, 0.25, seed=21,
                             window=((w, w), (w + N - 1, w + N - 1)))
    draws = iter([rng.random(N + 2 * w), rng.random(N + 2 * w)])
    err, ref = _truncated_vs_big(
        orc, N, w, lambda: orc.sigma_profile(N, w, orc.KIND_RANDOM, 2.0, draws=next(draws)),
        30, 160, u0)
    assert ref > 1e-2
    assert err < 1e-14, err


def test_reflectionless_3d_random_sigma(orc):
    """Thm 1.1 holds in any dimension: in 3D, with independent random damping per edge on
    all three axes, a pulse near a corner (it crosses an interface of every axis) matches an
    undamped box whose edges stay out of reach, to machine zero over the physical window."""
    N, w, steps = 16, 16, 16
    rng = np.random.default_rng(26)
    T = N + 2 * w
    sigs = [orc.sigma_profile(N, w, orc.KIND_RANDOM, 2.0, draws=rng.random(T)) for _ in range(3)]
    wl = wk.Workload("t", 3, (N, N, N), w, gaussians=[wk.Gaussian((w + 3.0, w + 12.5, w + 2.5), 2.0, 2.0)])
    u0 = wk.initial_field(wl)
    g = orc.Grid((T, T, T), 1.0, sigs)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    yn, _ = orc.rk4(g, y, steps, 0.5)
    M = 80
    off = (M - N) // 2
    ub = np.zeros((M, M, M))
    ub[off:off + N, off:off + N, off:off + N] = u0[w:w + N, w:w + N, w:w + N]
    gb = orc.Grid((M, M, M), 1.0, [np.zeros(M)] * 3)
    yb = gb.zeros_state()
    yb[0] = ub.reshape(-1)
    ybn, _ = orc.rk4(gb, yb, steps, 0.5, openmp=True)
    a = g.field(yn, 0)[w:w + N, w:w + N, w:w + N]
    big = gb.field(ybn, 0)
    b = big[off:off + N, off:off + N, off:off + N]
    beyond = big.copy()
    beyond[off:off + N, off:off + N, off:off + N] = 0.0
    assert np.abs(b).max() > 1e-2 and np.abs(beyond).max() > 1e-2   # part of the pulse has left
    assert np.abs(a - b).max() < 1e-14, np.abs(a - b).max()


def test_residual_waves_shrink_with_thickness(orc):
    """Sec. 1.1.4: residual waves shrink exponentially as the layer thickens linearly."""
    N = 24
    errs = []
    for w in (4, 8, 16):
        wl = wk.Workload("t", 2, (N, N), w, gaussians=[wk.Gaussian((w + 10.0, w + 12.0), 3.0, 1.0)])
        u0 = wk.initial_field(wl)
        e, _ = _truncated_vs_big(orc, N, w,
                                 lambda: orc.sigma_profile(N, w, orc.KIND_CONSTANT, 1.0),
                                 160, 24 + 2 * 100, u0)
        errs.append(e)
    assert errs[0] > 10 * errs[1] > 100 * errs[2], errs


# ----------------------------------------------------------------------------------
# Stability (Sec. 1.1.5): long runs with constant sigma = 2/h and random sigma in
# [0, 2/h] on a 20-cell layer keep the field bounded, and the energy in the physical
# domain decays.
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["constant", "random"])
def test_long_run_bounded_energy_decays(orc, kind):
    N, w = 16, 20
    rng = np.random.default_rng(22)
    if kind == "constant":
        sigs = [orc.sigma_profile(N, w, orc.KIND_CONSTANT, 2.0) for _ in range(2)]
    else:
        sigs = [orc.sigma_profile(N, w, orc.KIND_RANDOM, 2.0, draws=rng.random(N + 2 * w))
                for _ in range(2)]
    T = (N + 2 * w,) * 2
    g = orc.Grid(T, 1.0, sigs)
    wl = wk.Workload("t", 2, (N, N), w, gaussians=[wk.Gaussian((w + 8.0, w + 8.0), 2.0, 2.0)])
    y = g.zeros_state()
    y[0] = wk.initial_field(wl).reshape(-1)
    lo, hi = (w, w), (w + N - 1, w + N - 1)
    E0 = orc.energy(g, y, lo, hi)
    maxes = []
    for _ in range(20):
        y, _ = orc.rk4(g, y, 250, 0.5)
        maxes.append(np.abs(y).max())
    assert np.all(np.isfinite(y))
    assert max(maxes) < 10.0
    assert orc.energy(g, y, lo, hi) < 1e-8 * E0


# ----------------------------------------------------------------------------------
# Discrete adjoint: A^T against the dense transpose, and the dot-product identity
# <P^n x, z> = <x, (P^T)^n z> for the RK4 map; gradients against central differences
# (exact up to rounding because the misfit is quadratic in (U0, a)).
# ----------------------------------------------------------------------------------

def test_transpose_matches_dense(orc):
    rng = np.random.default_rng(23)
    for T, w, nd, h, wall in (((9,), 3, 1, 1.0, False), ((7, 8), 2, 2, 1.0, False), ((6, 5, 7), 2, 3, 1.0, False),
                              ((7, 8), 2, 2, 0.7, False), ((8, 7), 2, 2, 0.7, True)):
        sigs = [orc.sigma_profile(t - 2 * w, w, orc.KIND_RANDOM, 2.0 / h, draws=rng.random(t))
                for t in T]
        if wall:
            for sg in sigs:
                sg[-1] = 0.0
        g = orc.Grid(T, h, sigs, wall=wall)
        A = _dense_A(orc, g)
        N = A.shape[0]
        AT = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            AT[:, j] = orc.rhs_transpose(g, e).reshape(-1)
        assert np.abs(AT - A.T).max() < 1e-14


def test_adjoint_dot_product(orc):
    rng = np.random.default_rng(24)
    N, w = 8, 4
    sigs = [orc.sigma_profile(N, w, orc.KIND_POWER, 2.0, 2.0) for _ in range(2)]
    g = orc.Grid((N + 2 * w,) * 2, 1.0, sigs)
    x = _random_state(g, rng)
    z = _random_state(g, rng)
    n = 7
    Px, _ = orc.rk4(g, x, n, 0.5)
    PTz, _ = orc.adjoint(g, z, n, 0.5, n)
    lhs = float(np.sum(Px * z))
    rhs = float(np.sum(x * PTz))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_adjoint_dot_product_3d_random_sigma(orc):
    rng = np.random.default_rng(27)
    N, w = 4, 3
    T = N + 2 * w
    sigs = [orc.sigma_profile(N, w, orc.KIND_RANDOM, 2.0, draws=rng.random(T)) for _ in range(3)]
    g = orc.Grid((T, T, T), 1.0, sigs)
    x = _random_state(g, rng)
    z = _random_state(g, rng)
    n = 5
    Px, _ = orc.rk4(g, x, n, 0.4)
    PTz, _ = orc.adjoint(g, z, n, 0.4, n)
    lhs = float(np.sum(Px * z))
    rhs = float(np.sum(x * PTz))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_adjoint_gradients_vs_central_differences(orc):
    rng = np.random.default_rng(25)
    N, w = 12, 6
    sigs = [orc.sigma_profile(N, w, orc.KIND_POWER, 2.0, 2.0) for _ in range(2)]
    T = (N + 2 * w,) * 2
    g = orc.Grid(T, 1.0, sigs)
    dt, n = 0.5, 30
    f = 0.1
    src_xy = [(w + 3, w + 4), (w + 8, w + 7), (w + 5, w + 9)]
    src = {"idx": np.array([g.flat(c) for c in src_xy]), "amp": rng.uniform(-1, 1, 3),
           "f_peak": f, "t_delay": 1.5 / f}
    rec = np.array([g.flat((w + k, w + 1)) for k in range(0, N, 3)])
    u0 = np.zeros(g.n)
    u0[g.flat((w + 6, w + 6))] = 1.0
    u0[g.flat((w + 5, w + 6))] = 0.4
    d = rng.normal(scale=0.05, size=(n, len(rec)))

    def J(u0_, amp_):
        s = dict(src)
        s["amp"] = amp_
        y = g.zeros_state()
        y[0] = u0_
        _, tr = orc.rk4(g, y, n, dt, sources=s, receivers=rec)
        return 0.5 * np.sum((tr - d) ** 2), tr

    J0, tr = J(u0, src["amp"])
    yb = g.zeros_state()
    yb_out, gamp = orc.adjoint(g, yb, n, dt, n, sources=src, receivers=rec,
                               residual=(tr - d)[::-1].copy())
    eps = 1e-3
    for s_ in range(3):
        ap, am = src["amp"].copy(), src["amp"].copy()
        ap[s_] += eps
        am[s_] -= eps
        fd = (J(u0, ap)[0] - J(u0, am)[0]) / (2 * eps)
        assert abs(fd - gamp[s_]) < 1e-8 * max(abs(fd), 1e-6), (fd, gamp[s_])
    for v in (g.flat((w + 6, w + 6)), g.flat((w + 2, w + 3)), g.flat((w + 11, w + 1))):
        up, um = u0.copy(), u0.copy()
        up[v] += eps
        um[v] -= eps
        fd = (J(up, src["amp"])[0] - J(um, src["amp"])[0]) / (2 * eps)
        assert abs(fd - yb_out[0, v]) < 1e-8 * max(abs(fd), 1e-6), (fd, yb_out[0, v])


# ----------------------------------------------------------------------------------
# Gradient of the receiver misfit with respect to the edge damping sigma_a[e] (the
# supports of Phi/Psi held fixed): central differences of J(sigma), computed by forward
# runs only, against the reverse-stage-graph gradient.  J is smooth in every sigma_a[e]
# that stays nonzero, so the difference quotient agrees up to O(eps^2).
# ----------------------------------------------------------------------------------

def _grad_sigma_case(orc, N, w, steps, seed):
    rng = np.random.default_rng(seed)
    sig = [orc.sigma_profile(n, w, orc.KIND_RANDOM, 2.0, draws=rng.random(n + 2 * w)) for n in N]
    g = orc.Grid(tuple(n + 2 * w for n in N), 1.0, sig)
    y = g.zeros_state()
    y[0] = rng.normal(size=g.n)
    y[1] = 0.3 * rng.normal(size=g.n)
    rec = [g.flat(tuple(w + int(rng.integers(0, n)) for n in N)) for _ in range(3)]
    src = {"idx": [g.flat(tuple(w + n // 2 for n in N))], "amp": [0.7], "f_peak": 0.1, "t_delay": 10.0}
    tgt = 0.1 * rng.normal(size=(steps, len(rec)))
    return g, sig, y, rec, src, tgt


@pytest.mark.parametrize("N,w,steps", [((10, 9), 3, 25), ((5, 4, 6), 2, 12)])
def test_grad_sigma_matches_central_differences(orc, N, w, steps):
    g, sig, y, rec, src, tgt = _grad_sigma_case(orc, N, w, steps, seed=sum(N) + w)
    J, grad = orc.misfit_grad_sigma(g, y, steps, 0.5, rec, tgt, sources=src)
    assert J > 0

    def J_of(sigs):
        return orc.misfit_grad_sigma(orc.Grid(g.T, 1.0, sigs), y, steps, 0.5, rec, tgt, sources=src)[0]

    eps = 1e-5
    checked = 0
    for a in range(len(N)):
        T = g.T[a]
        for e in (0, 1, w - 2, T - 1, T - 2, T - w):
            e %= T
            if sig[a][e] == 0.0:
                assert grad[a][e] == 0.0
                continue
            sp = [s.copy() for s in sig]
            sm = [s.copy() for s in sig]
            sp[a][e] += eps
            sm[a][e] -= eps
            fd = (J_of(sp) - J_of(sm)) / (2 * eps)
            assert abs(grad[a][e] - fd) <= 1e-6 * max(abs(fd), 1e-3), (a, e, grad[a][e], fd)
            checked += 1
    assert checked >= 4


def test_grad_sigma_zero_on_physical_edges(orc):
    g, sig, y, rec, src, tgt = _grad_sigma_case(orc, (10, 9), 3, 10, seed=3)
    _, grad = orc.misfit_grad_sigma(g, y, 10, 0.5, rec, tgt, sources=src)
    for a in range(2):
        assert np.all(grad[a][sig[a] == 0.0] == 0.0)
        assert np.any(grad[a] != 0.0)


# ----------------------------------------------------------------------------------
# Layer backed by a reflecting wall (Sec. 1.1.4): every field is zero just beyond both
# ends of the box.  The interface still does not reflect, and the wave that comes back
# from the wall has crossed each layer edge there and back: its amplitude is the
# product of |rho(s, k)| / |rho(s, -conj k)| over the edges.
# ----------------------------------------------------------------------------------

def _wall_sigma(orc, n, w, kind, smax):
    s = orc.sigma_profile(n, w, kind, smax, 2.0)
    s[-1] = 0.0          # no edge from T-1 back to 0
    return s


def test_wall_layer_interface_does_not_reflect(orc):
    N, w = 32, 24
    wl = wk.Workload("t", 2, (N, N), w, gaussians=[wk.Gaussian((w + 7.0, w + 15.5), 3.0, 2.0)])
    u0 = wk.initial_field(wl)
    T = (N + 2 * w,) * 2
    g = orc.Grid(T, 1.0, [_wall_sigma(orc, N, w, orc.KIND_CONSTANT, 2.0) for _ in range(2)], wall=True)
    y = g.zeros_state()
    y[0] = u0.reshape(-1)
    yn, _ = orc.rk4(g, y, 40, 0.5)
    M = 160
    gb = orc.Grid((M, M), 1.0, [np.zeros(M), np.zeros(M)])
    off = (M - N) // 2
    ub = np.zeros((M, M))
    ub[off:off + N, off:off + N] = u0[w:w + N, w:w + N]
    yb = gb.zeros_state()
    yb[0] = ub.reshape(-1)
    ybn, _ = orc.rk4(gb, yb, 40, 0.5)
    a = g.field(yn, 0)[w:w + N, w:w + N]
    b = gb.field(ybn, 0)[off:off + N, off:off + N]
    assert np.abs(b).max() > 1e-2
    assert np.abs(a - b).max() < 1e-14


@pytest.mark.parametrize("kind,smax,kh", [(0, 0.04, 0.4), (1, 0.15, 0.7)])
def test_wall_backed_residual_matches_round_trip_factor(orc, kind, smax, kh):
    from paper_1804_01390_gb300 import _lib
    _lib.load()
    N, w, env = 300, 12, 25.0
    T = N + 2 * w
    sig = _wall_sigma(orc, N, w, kind, smax)
    j = np.arange(T)
    x0 = w + 0.7 * N
    G = np.exp(-0.5 * ((j - x0) / env) ** 2)
    wh = 2.0 * np.sin(kh / 2.0)
    U = G * np.cos(kh * (j - x0))
    V = wh * G * np.sin(kh * (j - x0))               # right-travelling, towards the wall
    steps = int(round(2.0 * (T - x0) / np.cos(kh / 2.0) / 0.5))
    amp = []
    for s_ in (sig, np.zeros(T)):
        g = orc.Grid((T,), 1.0, [s_], wall=True)
        y = g.zeros_state()
        y[0] = U
        y[1] = V
        yn, _ = orc.rk4(g, y, steps, 0.5)
        amp.append(np.abs(yn[0][w:w + N]).max())
    measured = amp[0] / amp[1]
    right = sig[w + N:T - 1]                          # the layer edges between the domain and the wall
    pred = _lib.pml_residual_factor(right, kh, wh, backed=True)
    assert 0.05 < measured < 0.9
    assert abs(measured - pred) <= 0.03 * pred, (measured, pred)


def test_wall_box_energy_decays(orc):
    N, w = 16, 20
    g = orc.Grid((N + 2 * w,) * 2, 1.0, [_wall_sigma(orc, N, w, orc.KIND_CONSTANT, 2.0) for _ in range(2)],
                 wall=True)
    wl = wk.Workload("t", 2, (N, N), w, gaussians=[wk.Gaussian((w + 8.0, w + 8.0), 2.0, 2.0)])
    y = g.zeros_state()
    y[0] = wk.initial_field(wl).reshape(-1)
    lo, hi = (w, w), (w + N - 1, w + N - 1)
    E0 = orc.energy(g, y, lo, hi)
    for _ in range(10):
        y, _ = orc.rk4(g, y, 250, 0.5)
    assert np.all(np.isfinite(y))
    assert orc.energy(g, y, lo, hi) < 1e-8 * E0
