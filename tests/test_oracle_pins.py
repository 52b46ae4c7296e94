"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of the sums, the paper's own analytic test (f == 1, Sec. 3.1),
textbook constants, library routines for special cases, and brute-force
dense solves at small N.  A plausible slip in the oracle (a dropped 1/N, a
wrong sign in G, an uncompensated y - x_k, a swapped index in Eq. p8) fails
at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------- exact constants

def test_pi_fixed_matches_textbook_hex(orc):
    hexdigits = _golden_lines("pi_hex.txt")[0][0]
    nbits = 4 * len(hexdigits)
    frac = orc.PI_FIXED - (3 << orc._PI_BITS)
    assert frac >> (orc._PI_BITS - nbits) == int(hexdigits, 16)
    assert float(Fraction(orc.PI_FIXED, 1 << orc._PI_BITS)) == math.pi


def test_bernoulli_matches_as64_table(orc):
    B = orc.bernoulli(20)
    for two_m, num, den in _golden_lines("bernoulli_as64.txt"):
        assert B[int(two_m)] == Fraction(int(num), int(den))
    assert all(B[k] == 0 for k in range(3, 21, 2))


def _pi_frac():
    from oracle import PI_FIXED, _PI_BITS
    return Fraction(PI_FIXED, 1 << _PI_BITS)


def test_bernoulli_bound_eq12(orc):
    """|B_2m| < 2 (2m)! / ((2 pi)^2m (1 - 2^(1-2m)))  (Eq. 12)."""
    B = orc.bernoulli(80)
    pi = _pi_frac()
    for m in range(1, 41):
        bound = Fraction(2 * math.factorial(2 * m)) / ((2 * pi) ** (2 * m) * (1 - Fraction(2) ** (1 - 2 * m)))
        assert abs(B[2 * m]) < bound


def _cot_series_tail(B, q, t):
    """2 sum_{m>q} |B_2m| t^(2m-1)/(2m)! (200 terms, exact coefficients)."""
    s = 0.0
    for m in range(q + 1, q + 60):
        s += float(abs(B[2 * m]) / math.factorial(2 * m)) * t ** (2 * m - 1)
    return 2.0 * s


@pytest.mark.parametrize("q", [2, 4, 8, 11, 14, 20])
def test_series_eq10_eq11_truncation(orc, q):
    """Eq. 10 truncated after q terms differs from cot(t/2) by < 2 eps_q on |t|<=pi,
    Eq. 11 (the tan series) by < 2 * (2 eps_q) on |t|<=pi/2  (Eq. p14)."""
    B = orc.bernoulli(2 * q + 130)
    eps_q = 2.0 ** (1 - 2 * q) / (3 * math.pi * (1 - 2.0 ** (-2 * q - 1)))
    ts = np.linspace(0.25, math.pi, 200)
    worst1 = worst2 = 0.0
    for t in ts:
        s1 = 2.0 / t - 2.0 * sum(float(abs(B[2 * m]) / math.factorial(2 * m)) * t ** (2 * m - 1)
                                  for m in range(1, q + 1))
        worst1 = max(worst1, abs(1.0 / math.tan(t / 2) - s1))
        t2 = t / 2
        s2 = -2.0 * sum(float((2 ** (2 * m) - 1) * abs(B[2 * m]) / math.factorial(2 * m)) * t2 ** (2 * m - 1)
                        for m in range(1, q + 1))
        worst2 = max(worst2, abs(-math.tan(t2 / 2) - s2))
    # the series themselves (and the bound) hold: the residual is the tail
    assert worst1 < 2 * eps_q + 1e-13
    assert worst2 < 2 * 2 * eps_q + 1e-13
    # the bound is not vacuous: the tail at t = pi is within a factor ~2 of it
    assert _cot_series_tail(B, q, math.pi) > 0.3 * eps_q


# ------------------------------------------------------------- forward sums

def _exact_expi(m, y):
    """e^{i m y} with m*y reduced mod 2 pi in exact rational arithmetic."""
    pi = _pi_frac()
    a = Fraction(m) * Fraction(y)
    r = a - 2 * pi * math.floor(a / (2 * pi))
    r = float(r)
    return complex(math.cos(r), math.sin(r))


@pytest.mark.parametrize("N", [8, 256, 1 << 16, 1000])
def test_nudft_reproduces_single_mode(orc, N):
    """c = e_m gives g_j = e^{i m y_j} exactly (band-limited series, Eq. p1)."""
    y = workloads.points("uniform", 64 if N < 65536 else 8, seed=3)
    for m in sorted({0, 1, N // 3, N - 1}):
        c = np.zeros(N, complex)
        c[m] = 1.0
        g = orc.nudft_fwd(c, y)
        ref = np.array([_exact_expi(m, v) for v in y])
        assert np.abs(g - ref).max() < 4e-16 * max(1, 8)


@pytest.mark.parametrize("N", [8, 64, 1024, 4096, 12, 100, 1000, 3 * 1024])
def test_kernel_form_constant_function(orc, N):
    """The paper's analytic test (Sec. 3.1): f == 1 gives g_j = 1 exactly, for
    random y and for y on or next to grid points (Eq. p4 with the 1/N of p5);
    the identity holds for every grid size N, powers of two or not."""
    L = N.bit_length()
    y = workloads.points("uniform", 200, seed=L)
    k = np.arange(0, N, max(1, N // 16))
    xk = k * (2 * math.pi / N)
    near = np.concatenate([xk, np.nextafter(xk, 10.0), np.nextafter(xk[1:], -10.0)])
    y = np.concatenate([y, near, [0.0]])
    y = y[(y >= 0) & (y < 2 * math.pi)]
    g = orc.kernel_fwd(np.ones(N, complex), y)
    assert np.abs(g - 1.0).max() < 1e-14


def _exact_cot_half(N, y):
    """N cot(N y / 2) with N y / 2 reduced modulo pi into [-pi/2, pi/2] in
    exact rationals (so a result near a pole keeps its relative precision)."""
    pi = _pi_frac()
    a = Fraction(N) * Fraction(y) / 2
    r = float(a - pi * round(a / pi))
    return N / math.tan(r)


@pytest.mark.parametrize("N", [16, 1024, 4096, 12, 1000, 3 * 1024])
def test_cot_sum_closed_form(orc, N):
    """sum_k cot((y - 2 pi k/N)/2) = N cot(N y/2): pins G and the compensated
    difference y - x_k (a double-double 2 pi / N for any N), including y
    within an ulp of a grid point."""
    y = workloads.points("uniform", 100, seed=N)
    k = np.arange(1, N, max(1, N // 8))
    xk = k * (2 * math.pi / N)
    y = np.concatenate([y, np.nextafter(xk, 10.0), np.nextafter(xk, -10.0)])
    h = orc.cot_sum(np.ones(N), y)
    ref = np.array([_exact_cot_half(N, v) for v in y])
    assert np.all(np.abs(h - ref) <= 1e-13 * np.maximum(np.abs(ref), N))


@pytest.mark.parametrize("N,M", [(64, 50), (1024, 300), (4096, 64), (100, 80), (1000, 300)])
def test_two_forward_routes_agree(orc, N, M):
    """Direct NUDFT (Eq. p1) and the factored kernel form (Eq. p2/p4) agree."""
    c = workloads.coeffs(N, seed=N)
    y = workloads.points("uniform", M, seed=M)
    g1 = orc.nufft_fwd(c, y, route="nudft")
    g2 = orc.nufft_fwd(c, y, route="kernel")
    assert orc.rel_l2(g2, g1) < 1e-13


@pytest.mark.parametrize("N", [8, 32, 64, 12, 30])
def test_dense_kernel_matrix(orc, N):
    """Columns of the factored form equal the geometric sum of Eq. p2 and the
    Dirichlet closed form (reading c1: F_j carries the 1/N)."""
    M = 40
    y = workloads.points("uniform", M, seed=N + 1)
    K = np.empty((M, N), complex)
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1.0
        K[:, k] = orc.kernel_fwd(e, y)
    x = 2 * np.pi * np.arange(N) / N
    n = np.arange(N)
    Kp2 = np.exp(1j * (y[:, None, None] - x[None, :, None]) * n[None, None, :]).sum(-1) / N
    assert np.abs(K - Kp2).max() < 1e-13
    t = y[:, None] - x[None, :]
    Kd = np.exp(1j * (N - 1) * t / 2) * np.sin(N * t / 2) / np.sin(t / 2) / N
    assert np.abs(K - Kd).max() < 1e-12


def test_adjoint_dot_product(orc):
    """<A c, g> = <c, A^H g> for the direct forward and adjoint, and the
    factored adjoint route agrees with the direct one."""
    N, M = 512, 300
    c = workloads.coeffs(N, seed=5)
    g = workloads.samples(M, seed=6)
    y = workloads.points("uniform", M, seed=7)
    Ac = orc.nudft_fwd(c, y)
    Ahg = orc.nudft_adj(g, y, N)
    lhs, rhs = np.vdot(g, Ac), np.vdot(Ahg, c)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    assert orc.rel_l2(orc.nufft_adj(g, y, N, route="kernel"), Ahg) < 1e-13


def test_fft_matches_dft_and_numpy(orc):
    for N in (8, 64, 1024):
        x = workloads.coeffs(N, seed=N)
        assert orc.rel_l2(orc.fft(x, -1), np.fft.fft(x)) < 1e-14
        assert orc.rel_l2(orc.fft(x, +1), np.fft.ifft(x) * N) < 1e-14
        assert orc.rel_l2(orc.dft(x, -1), np.fft.fft(x)) < 1e-14


# ------------------------------------------------------------- threshold error (Sec. 3.1)

def test_straightforward_method_close_to_compensated_at_small_n(orc):
    """The plain-binary64 Eq. p4 product (the paper's straightforward method)
    equals the compensated oracle to within its own rounding: each term's
    uncompensated difference y - k fl(2 pi/N) is off by at most ~2 ulp(2 pi),
    which moves K_jk by at most that times |dK/dt| ~ 1/(N t^2) -- small for
    points away from the grid, as here."""
    N, M = 64, 200
    y = workloads.rng(3).uniform(0, 2 * math.pi, M)
    x = 2 * math.pi * np.arange(N) / N
    dist = np.abs(np.angle(np.exp(1j * (y[:, None] - x[None, :])))).min(1)
    y = y[dist > 1e-3]
    f = workloads.coeffs(N, seed=4)
    gp = orc.kernel_fwd_plain(f, y)
    gc = orc.kernel_fwd(f, y)
    bound = 4 * 2.0 ** -52 * 2 * math.pi / (N * dist[dist > 1e-3] ** 2) * np.abs(f).sum() + 1e-13
    assert np.all(np.abs(gp - gc) <= bound)
    # the f = 1 sum reproduces 1 up to the same rounding
    g1 = orc.kernel_fwd_plain(np.ones(N, complex), y)
    assert np.abs(g1 - 1).max() < 1e-11


def test_threshold_error_grows_with_n(orc):
    """The paper's threshold phenomenon (Sec. 3.1): the straightforward
    method's error for f = 1 grows with N, while the compensated oracle stays
    at the rounding level; and the committed table (written by
    oracle/eps_threshold.py) reproduces for the small sizes, within a factor
    2 (its maxima depend on single roundings of libm)."""
    rows = [list(map(float, r)) for r in _golden_lines("eps_threshold_straightforward.txt")]
    table = {int(r[0]): r for r in rows}
    assert table[1 << 20][2] > 100 * table[1 << 8][2]
    assert all(r[6] <= 32 and r[7] <= 24 for r in rows)           # p_th, q_th bounded
    assert table[1 << 20][7] < table[1 << 8][7]                     # q_th decays
    from oracle import eps_threshold
    for L in (6, 9, 12):
        N, nt, e1, er = eps_threshold.measure(L, 1024)
        assert 0.5 * table[N][2] <= e1 <= 2.0 * table[N][2]
        g = orc.kernel_fwd(np.ones(N, complex), workloads.points("uniform", N, seed=500 + L),
                           workloads.sample_index(N, 1024, seed=L))
        assert np.abs(g - 1).max() < 1e-13
        if L >= 9:
            assert e1 > 1e-11


# ------------------------------------------------------------- inverse

@pytest.mark.parametrize("N", [16, 256, 12, 100])
def test_logsin_equispaced_closed_form(orc, N):
    """y_l = 2 pi l/N + phi: prod_l 2 sin((x - y_l)/2) = +-2 sin(N (x - phi)/2)
    and prod_{l!=j} 2 sin((y_j - y_l)/2) = +-N, which pin the log-sums and the
    sign counts behind C_k and D_j (Eq. p8)."""
    phi = 0.37 * 2 * math.pi / N
    y = 2 * math.pi * np.arange(N) / N + phi
    lamC, nC = orc.logsin_C(y, N)
    assert np.abs(lamC - math.log(2 * abs(math.sin(N * phi / 2)))).max() < 1e-12
    assert np.array_equal(nC, N - np.arange(N))
    lamD, nD = orc.logsin_D(y)
    assert np.abs(lamD + math.log(N)).max() < 1e-12
    assert np.array_equal(nD, N - 1 - np.arange(N))


@pytest.mark.parametrize("N,jit", [(32, 0.1), (128, 0.1), (256, 0.1), (64, 0.4), (30, 0.1),
                                   (100, 0.1)])
def test_inverse_round_trip_and_dense_solve(orc, N, jit):
    """At M = N the Lagrange form (Eq. p6, p8) inverts the forward transform:
    inufft(nudft_fwd(c)) = c, equal to a dense LU solve of A c = g."""
    y = workloads.points("jitter", N, N, seed=N, jitter=jit)
    c = workloads.coeffs(N, seed=N + 3)
    g = orc.nudft_fwd(c, y)
    c2 = orc.inufft(g, y, N)
    A = np.exp(1j * np.outer(y, np.arange(N)))
    cs = np.linalg.solve(A, g)
    tol = 1e-12 if jit <= 0.1 else 1e-10
    assert orc.rel_l2(c2, c) < tol
    assert orc.rel_l2(c2, cs) < tol


@pytest.mark.parametrize("N,kind", [(128, "jitter"), (16, "clustered")])
def test_inverse_modulus_sum_is_dense_lagrange_matrix(orc, N, kind):
    """sum_j |L_kj| |g_j| of the Lagrange form equals |B A^-1| |g| for the
    dense matrices A_jn = e^(i n y_j), B_kn = e^(i n x_k) built by numpy (L
    maps the samples to the grid values of their band-limited interpolant),
    and the signed sum is (B A^-1) g.  The clustered case is small (cond(A)
    ~ 7e5) so that numpy's dense inverse is itself accurate to ~1e-10."""
    y = workloads.points(kind, N, N if kind == "jitter" else None, seed=N, jitter=0.4)
    y = np.sort(y)
    g = workloads.samples(N, seed=3)
    n = np.arange(N)
    A = np.exp(1j * np.outer(y, n))
    Bm = np.exp(1j * np.outer(2 * np.pi * n / N, n))
    L = Bm @ np.linalg.inv(A)
    a_ref = np.abs(L) @ np.abs(g)
    a = orc.inverse_absf(g, y, N)
    tol = 1e-13 if kind == "jitter" else 1e-9
    assert np.abs(a - a_ref).max() <= tol * a_ref.max()
    f = orc.inverse_f(g, y, N)
    assert np.abs(f - L @ g).max() <= tol * a_ref.max()


def test_inverse_exact_hit(orc):
    """y_0 = 0 = x_0 exactly: C_0 = 0 and f_0 = g_0 (reading c7)."""
    N = 64
    y = workloads.points("jitter", N, N, seed=9, jitter=0.1)
    y[0] = 0.0
    c = workloads.coeffs(N, seed=1)
    g = orc.nudft_fwd(c, y)
    f = orc.inverse_f(g, y, N)
    assert f[0] == g[0]
    assert orc.rel_l2(orc.fft(f, -1) / N, c) < 1e-12


# ------------------------------------------------------------- exact grid / binning

def test_exact_grid_generic_points(orc):
    N, B = 1 << 12, 1 << 7
    y = workloads.points("uniform", 500, seed=11)
    leaf, k0, delta = orc.exact_grid(y, N, B)
    Y = y * N / (2 * math.pi)
    assert np.abs((k0 + delta) - Y).max() < 1e-9
    assert np.array_equal(leaf, np.floor((k0 + delta) / (N // B)).astype(np.int64) % B)
    assert np.all(np.abs(delta) <= 0.5)


def test_exact_grid_boundaries_and_hits(orc):
    N, B = 1 << 10, 1 << 5
    s = N // B
    b = np.arange(B)
    edge = b * (2 * math.pi / B)
    below = np.nextafter(edge[1:], -10.0)
    above = np.nextafter(edge, 10.0)
    y = np.concatenate([[0.0], below, above])
    leaf, k0, delta = orc.exact_grid(y, N, B)
    assert leaf[0] == 0 and k0[0] == 0 and delta[0] == 0.0
    # one ulp below a leaf edge lies in the leaf to the left, one above in the leaf
    assert np.array_equal(leaf[1:B], b[:-1])
    assert np.array_equal(leaf[B:], b)
    # the nearest grid point of an edge is the edge's grid index, |delta| tiny
    assert np.array_equal(k0[1:B], (b[1:] * s) % N)
    assert np.abs(delta[1:]).max() < 1e-12


def test_binning_is_stable_counting_sort(orc):
    """Leaves in order; inside a leaf, the points keep their original order
    (a stable counting sort by leaf, Sec. 2.1); every point's grid coordinate
    y N / (2 pi) = k0 + delta lies in its leaf's half-open arc; the result
    equals numpy's stable argsort of the exact leaf index and a plain Python
    bucket sort of the points."""
    N, B = 1 << 10, 1 << 6
    s = N // B
    y = workloads.points("clustered", 3000, seed=4)
    perm, start, leaf = orc.binning(y, N, B)
    _, k0, delta = orc.exact_grid(y, N, B)
    assert np.array_equal(np.sort(perm), np.arange(y.size))
    assert np.all(np.diff(leaf[perm]) >= 0)
    buckets = [[] for _ in range(B)]
    for j, b in enumerate(leaf.tolist()):
        buckets[b].append(j)
    assert np.array_equal(perm, np.array([j for bk in buckets for j in bk]))
    for bb in range(B):
        seg = perm[start[bb]:start[bb + 1]]
        assert np.all(leaf[seg] == bb)
        assert np.all(np.diff(seg) > 0)  # original order inside the leaf
        krel = (k0[seg] - bb * s) % N
        Y = bb * s + krel + delta[seg]
        assert np.all((Y >= bb * s) & (Y < bb * s + s))
    assert start[0] == 0 and start[-1] == y.size
    # the leaf of an ordinary (non-edge) point is what floating point says
    Yf = y * (N / (2 * math.pi)) / s
    safe = np.abs(Yf - np.round(Yf)) > 1e-6
    assert np.array_equal(leaf[safe], np.floor(Yf[safe]).astype(np.int64) % B)


# ------------------------------------------------------------- density-compensation network

def test_mlp_oracle_gradient_matches_finite_differences():
    """The FP64 reference gradient of the DCF network equals central finite
    differences of its loss (pins the hand-written chain rule)."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.NPARAM) * 0.3
    X = rng.standard_normal((40, 8))
    t = rng.standard_normal(40)
    g, _ = mlp.grad(p, X, t)
    for k in list(range(0, 512, 97)) + [512, 600, 4000, 4672, 4700, 4736, 4799, 4800]:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss(pp, X, t) - mlp.loss(pm, X, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), k


def test_mlp_oracle_forward_closed_forms():
    """Forward pass of the DCF network at weights where it has a closed form:
    with W1 = W2 = 0 the output is softplus(W3 . gelu(b2) + b3), and
    gelu(x) = x Phi(x) with the tabulated normal distribution function
    (tests/golden/normal_cdf_as26.txt); softplus(0) = log 2 and
    softplus(log(e - 1)) = 1.  One nonzero W2[u, v] checks that the hidden
    layer is h1 @ W2^T (not W2 h1 transposed) and that the layers nest."""
    from oracle import mlp
    table = {float(x): float(v) for x, v in _golden_lines("normal_cdf_as26.txt")}
    X = np.random.default_rng(1).standard_normal((5, 8))
    base = np.zeros(mlp.NPARAM)
    q = mlp.unpack(base)  # views into base
    # zero network: w = softplus(0) = log 2 for every point
    assert np.allclose(mlp.forward(base, X), math.log(2.0), rtol=0, atol=1e-15)
    # output bias alone
    q["b3"] = math.log(math.e - 1.0)
    p = base.copy()
    p[-1] = math.log(math.e - 1.0)
    assert np.allclose(mlp.forward(p, X), 1.0, rtol=0, atol=1e-15)
    # W1 = W2 = 0: z = sum_u W3_u gelu(b2_u) + b3, gelu from the table
    p = np.zeros(mlp.NPARAM)
    pq = mlp.unpack(p)
    pq["b2"][:3] = list(table)           # 0.5, 1.0, 2.0
    pq["W3"][:3] = [1.0, -2.0, 0.5]
    z = sum(wt * x * table[x] for wt, x in zip([1.0, -2.0, 0.5], table))
    assert np.allclose(mlp.forward(p, X), math.log1p(math.exp(z)), rtol=1e-14, atol=0)
    # one path through W2: b1_v = 1, W2[u, v] = 1, W3_u = 1 (u != v)
    u, v = 7, 40
    p = np.zeros(mlp.NPARAM)
    pq = mlp.unpack(p)
    pq["b1"][v] = 1.0
    pq["W2"][u, v] = 1.0
    pq["W3"][u] = 1.0
    h1 = 1.0 * table[1.0]
    h2 = h1 * 0.5 * (1.0 + math.erf(h1 / math.sqrt(2.0)))
    assert np.allclose(mlp.forward(p, X), math.log1p(math.exp(h2)), rtol=1e-14, atol=0)
    # the input layer reads feature k through W1[u, k]
    p = np.zeros(mlp.NPARAM)
    pq = mlp.unpack(p)
    pq["W1"][3, 5] = 1.0
    pq["W2"][0, 3] = 1.0
    pq["W3"][0] = 1.0
    X2 = np.zeros((3, 8))
    X2[:, 5] = [0.5, 1.0, 2.0]
    a1 = X2[:, 5]
    h1 = a1 * np.array([table[x] for x in (0.5, 1.0, 2.0)])
    h2 = h1 * 0.5 * (1.0 + np.array([math.erf(x / math.sqrt(2.0)) for x in h1]))
    assert np.allclose(mlp.forward(p, X2), np.log1p(np.exp(h2)), rtol=1e-14, atol=0)


def _frobenius_dcf(y, N):
    """Density-compensation weights minimising ||A^H W A - I||_F (reading c13)
    by a dense linear least-squares solve over the M columns vec(a_j a_j^H),
    a_j the j-th row of A_jn = e^{i n y_j}; no kernel formula involved."""
    A = np.exp(1j * np.outer(y, np.arange(N)))
    cols = np.stack([np.outer(A[j].conj(), A[j]).ravel() for j in range(y.size)], axis=1)
    rhs = np.eye(N).ravel().astype(complex)
    w, *_ = np.linalg.lstsq(np.vstack([cols.real, cols.imag]),
                            np.concatenate([rhs.real, rhs.imag]), rcond=None)
    return w


def test_dcf_fixed_point_equispaced_closed_form():
    """On equispaced points with M a multiple of N every row of |D_N|^2 sums
    to N M, so the fixed point is w = 1 / M everywhere: log(w / mean w) = 0."""
    from oracle import mlp
    for N, M in ((16, 64), (32, 96)):
        y = 2 * np.pi * np.arange(M) / M + 0.1
        y = np.mod(y, 2 * np.pi)
        assert np.abs(mlp.dcf_fixed_point(y, N, iters=50)).max() < 1e-12


def _frobenius_objective(y, N, w):
    A = np.exp(1j * np.outer(y, np.arange(N)))
    return float(np.linalg.norm((A.conj().T * w) @ A - np.eye(N)))


def test_dcf_fixed_point_is_frobenius_optimum():
    """The fixed point solves the normal equations of min ||A^H W A - I||_F
    (reading c13).  With M <= 2N - 1 the minimiser is unique and, on these
    jittered points, positive: the iteration converges to it (up to the
    normalisation to mean 1), compared with a dense least-squares solve that
    never forms |D_N|^2.  With M > 2N - 1 the minimiser is not unique; the
    objective at the fixed point, rescaled, still equals the least-squares
    minimum."""
    from oracle import mlp
    rng = np.random.default_rng(21)
    N, M = 32, 60
    y = np.sort(np.mod(2 * np.pi * np.arange(M) / M + rng.uniform(-0.3, 0.3, M) * 2 * np.pi / M,
                       2 * np.pi))
    w_ref = _frobenius_dcf(y, N)
    assert np.all(w_ref > 0)
    lw = mlp.dcf_fixed_point(y, N, iters=3000)
    assert np.abs(lw - np.log(w_ref / w_ref.mean())).max() < 1e-9
    # a slip that keeps translation invariance (|D_N| not squared) is caught
    t = y[:, None] - y[None, :]
    sn = np.sin(0.5 * t)
    K1 = np.abs(np.sin(0.5 * N * t) / np.where(np.abs(sn) < 1e-12, 1.0, sn))
    K1[np.abs(sn) < 1e-12] = N
    w1 = np.ones(M)
    for _ in range(3000):
        w1 = w1 * N / (K1 @ w1)
    assert np.abs(np.log(w1 / w1.mean()) - np.log(w_ref / w_ref.mean())).max() > 1e-3
    # rank-deficient case: same optimal objective
    N, M = 16, 48
    y = np.sort(np.mod(2 * np.pi * np.arange(M) / M + rng.uniform(-0.3, 0.3, M) * 2 * np.pi / M,
                       2 * np.pi))
    w_ref = _frobenius_dcf(y, N)
    w = np.exp(mlp.dcf_fixed_point(y, N, iters=3000))
    A = np.exp(1j * np.outer(y, np.arange(N)))
    Bw = (A.conj().T * w) @ A
    sc = np.trace(Bw).real / np.linalg.norm(Bw) ** 2  # best scale of the normalised weights
    assert _frobenius_objective(y, N, sc * w) <= _frobenius_objective(y, N, w_ref) * (1 + 1e-8)


# ------------------------------------------------------------- symmetries of the sums

@pytest.mark.parametrize("N,m", [(64, 5), (256, 77), (1024, 1000)])
def test_nudft_grid_shift_theorem(orc, N, m):
    """Eq. p1 under a shift of the points by m grid steps: g(y + 2 pi m / N)
    equals the sum with c_n e^(2 pi i n m / N) at y (both routes), checked on
    points whose shifted copies stay inside [0, 2 pi).  The shifted points are
    binary64 roundings of y + 2 pi m / N (|error| <= 2^-50 2 pi), which moves
    term n by a phase of at most n times that: the bound below."""
    rng = np.random.default_rng(N + m)
    h = 2 * math.pi / N
    y = rng.uniform(0, 2 * math.pi - (m + 1) * h, 200)
    c = workloads.coeffs(N, seed=m)
    cs = c * np.exp(2j * math.pi * np.arange(N) * m / N)
    ys = y + m * h
    for route in ("nudft", "kernel"):
        lhs = orc.nufft_fwd(c, ys, route=route)
        rhs = orc.nufft_fwd(cs, y, route=route)
        assert orc.rel_l2(lhs, rhs) < N * 2.0 ** -50 * 2 * math.pi + 1e-14, route


@pytest.mark.parametrize("N", [32, 512])
def test_nudft_reflection(orc, N):
    """Eq. p1 at 2 pi - y is the conjugate sum: sum conj(c_n) e^(i n (2 pi - y))
    = conj(sum c_n e^(i n y)); the adjoint obeys the same reflection."""
    rng = np.random.default_rng(N)
    y = rng.uniform(1e-3, 2 * math.pi - 1e-3, 300)
    c = workloads.coeffs(N, seed=3)
    g = workloads.samples(300, seed=4)
    assert orc.rel_l2(orc.nudft_fwd(np.conj(c), 2 * math.pi - y),
                      np.conj(orc.nudft_fwd(c, y))) < 1e-13
    assert orc.rel_l2(orc.nudft_adj(np.conj(g), 2 * math.pi - y, N),
                      np.conj(orc.nudft_adj(g, y, N))) < 1e-13


def test_adjoint_is_conjugate_transpose_of_dense_matrix(orc):
    """The adjoint route equals A^H g for the dense matrix A_jn = e^(i n y_j)
    built by numpy (brute force at small N)."""
    N, M = 64, 70
    rng = np.random.default_rng(9)
    y = rng.uniform(0, 2 * math.pi, M)
    g = workloads.samples(M, seed=10)
    A = np.exp(1j * np.outer(y, np.arange(N)))
    for route in ("nudft", "kernel"):
        assert orc.rel_l2(orc.nufft_adj(g, y, N, route=route), A.conj().T @ g) < 1e-12, route
