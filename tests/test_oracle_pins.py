"""Pins for the CPU oracle: each test checks it against something other than
itself -- a closed form, an exact rational computation, an invariant of the
scheme, a published value, or the paper's own equations -- so that a dropped
term, a wrong sign, a wrong index or a transposed operand fails at least one.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1602_07558_gb300 import inputs

EPS = np.finfo(np.float64).eps
MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------- heat

@pytest.mark.parametrize("T", [64, 512])
def test_heat_single_fourier_mode_decays_by_exact_factor(oracle_lib, T):
    """A single mode sin(2 pi 3 x/64) sin(2 pi 5 y/64) is an eigenvector of the
    5-point forward-Euler scheme with factor g = 1 - 4 r (sin^2(pi p/N) + sin^2(pi q/N))
    per step (discrete Fourier analysis); the oracle must follow g^T up to rounding,
    which the max-norm-stable scheme (r = 0.2 <= 1/4) does not amplify."""
    n, p, q, r = 64, 3, 5, 0.2
    u0 = inputs.fourier_mode(n, n, p, q)
    g = 1.0 - 4.0 * r * (np.sin(np.pi * p / n) ** 2 + np.sin(np.pi * q / n) ** 2)
    uT = oracle_lib.heat(u0, r, T)
    err = np.max(np.abs(uT - g ** T * u0))
    assert err <= 4 * T * EPS * np.max(np.abs(u0))
    # the decayed amplitude itself (not only the error) is as predicted
    assert np.max(np.abs(uT)) == pytest.approx(g ** T * np.max(np.abs(u0)), rel=1e-9)


def test_heat_conserves_the_grid_sum(oracle_lib):
    """Sum over the periodic grid of (u_E + u_S + u_W + u_N - 4u) is zero, so the
    sum is conserved up to rounding."""
    u0 = inputs.uniform(48, 40, seed=7)
    T = 200
    uT = oracle_lib.heat(u0, 0.2, T)
    assert abs(uT.sum() - u0.sum()) <= T * u0.size * 4 * EPS
    assert not np.allclose(uT, u0)          # it did diffuse


@pytest.mark.parametrize("nx,ny,T", [(4, 4, 12), (6, 8, 10)])
def test_heat_matches_exact_rational_arithmetic(oracle_lib, nx, ny, T):
    """Brute force with exact rationals (r taken as the exact value of the double
    0.2): the oracle differs only by its rounding."""
    rng = np.random.default_rng(11)
    u0 = rng.integers(-16, 17, size=(ny, nx)) / 16.0
    r = Fraction(0.2)
    u = [[Fraction(float(u0[j, i])) for i in range(nx)] for j in range(ny)]
    for _ in range(T):
        u = [[u[j][i] + r * (u[j][(i + 1) % nx] + u[(j + 1) % ny][i] + u[j][(i - 1) % nx]
                             + u[(j - 1) % ny][i] - 4 * u[j][i])
              for i in range(nx)] for j in range(ny)]
    exact = np.array([[float(v) for v in row] for row in u])
    got = oracle_lib.heat(u0, 0.2, T)
    assert np.max(np.abs(got - exact)) <= T * 8 * EPS * np.max(np.abs(u0))


def test_heat_impulse_response_is_the_five_point_stencil(oracle_lib):
    """One step from a unit impulse: 1 - 4r at the centre, r at the 4 edge
    neighbours, exactly 0 at the diagonals and everywhere else."""
    u0 = np.zeros((9, 11))
    u0[4, 6] = 1.0
    u1 = oracle_lib.heat(u0, 0.2, 1)
    expect = np.zeros_like(u0)
    expect[4, 6] = 1.0 - 4.0 * 0.2
    for dj, di in [(0, 1), (0, -1), (1, 0), (-1, 0)]:
        expect[4 + dj, 6 + di] = 0.2
    assert np.array_equal(u1, expect)


def test_heat_is_translation_and_mirror_equivariant(oracle_lib):
    """The periodic scheme commutes with shifts and (by commutativity of each
    rounded addition) with mirroring in x and y, bit for bit."""
    u0 = inputs.uniform(20, 12, seed=3)
    uT = oracle_lib.heat(u0, 0.2, 9)
    shifted = oracle_lib.heat(np.roll(u0, (5, -7), axis=(0, 1)), 0.2, 9)
    assert np.array_equal(shifted, np.roll(uT, (5, -7), axis=(0, 1)))
    sq = inputs.uniform(16, 16, seed=4)
    assert np.array_equal(oracle_lib.heat(sq.T, 0.2, 7), oracle_lib.heat(sq, 0.2, 7).T)


# --------------------------------------------------------------------- increment

def test_increment_worked_example(oracle_lib):
    """Section 3.1: u^0 = 1 everywhere and St: u <- u + 1 gives 1 + T after T steps."""
    u = oracle_lib.increment(np.ones((8, 8)), 7)
    assert np.all(u == 8.0)


# -------------------------------------------------------------------------- hash

def test_mix64_is_splitmix64(oracle_lib):
    """SplitMix64 seeded with 0 (state advanced by the golden gamma, then the
    output function) has the published first outputs below."""
    golden = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [oracle_lib.mix64((k * golden) & MASK64) for k in (1, 2, 3)]
    assert got == expect


@pytest.mark.parametrize("s", [1, 2, 3])
def test_hash_domain_of_influence_is_the_9_point_square(oracle_lib, s):
    """Changing one word changes, after s sub-steps, exactly the points within
    Chebyshev distance s (the domain of influence of a 9-point radius-1 stencil,
    Section 2 and Section 3), with periodic wrap."""
    u0 = inputs.random_words(24, 20, seed=5)[0]
    u1 = u0.copy()
    j0, i0 = 1, 22                       # near two edges: exercises the wrap
    u1[j0, i0] ^= np.uint64(1 << 17)
    a, b = oracle_lib.hash_op(u0, s), oracle_lib.hash_op(u1, s)
    changed = a != b
    jj, ii = np.meshgrid(np.arange(20), np.arange(24), indexing="ij")
    dj = np.minimum((jj - j0) % 20, (j0 - jj) % 20)
    di = np.minimum((ii - i0) % 24, (i0 - ii) % 24)
    assert np.array_equal(changed, np.maximum(dj, di) <= s)


def test_hash_is_translation_equivariant_and_depends_on_the_substep(oracle_lib):
    u0 = inputs.random_words(16, 12, seed=6)[0]
    a = oracle_lib.hash_op(u0, 4, substep0=10)
    b = oracle_lib.hash_op(np.roll(u0, (3, 5), axis=(0, 1)), 4, substep0=10)
    assert np.array_equal(b, np.roll(a, (3, 5), axis=(0, 1)))
    c = oracle_lib.hash_op(u0, 4, substep0=11)
    assert np.all(a != c)


# ---------------------------------------------------------------------- leveltag

def test_leveltag_counts_levels_and_poisons_the_domain_of_influence(oracle_lib):
    u = oracle_lib.leveltag(np.full((10, 12), 3.0), 6)
    assert np.all(u == 9.0)
    u0 = np.zeros((10, 12))
    u0[5, 0] = 1.0                       # one point at the wrong level
    u2 = oracle_lib.leveltag(u0, 2)
    jj, ii = np.meshgrid(np.arange(10), np.arange(12), indexing="ij")
    dist = np.maximum(np.abs(jj - 5), np.minimum(ii, 12 - ii))
    assert np.array_equal(np.isnan(u2), dist <= 2)
    assert np.all(u2[dist > 2] == 2.0)


# ------------------------------------------------------------------------- wide2

def test_wide2_impulse_response(oracle_lib):
    """Eq. (complex_step) on a unit impulse: -4 at the centre, +1 two points away
    along each axis (modulo 2^64)."""
    u0 = np.zeros((9, 10), dtype=np.uint64)
    u0[4, 5] = 1
    u1 = oracle_lib.wide2(u0, 1)
    expect = np.zeros_like(u0)
    expect[4, 5] = np.uint64((1 << 64) - 4)
    for dj, di in [(0, 2), (0, -2), (2, 0), (-2, 0)]:
        expect[4 + dj, 5 + di] = 1
    assert np.array_equal(u1, expect)


def test_wide2_equals_the_two_substep_decomposition(oracle_lib):
    """Eqs. (substep1)-(substep2): pushing (u, u_W, u_E, u_N, u_S) in a first
    radius-1 sub-step and combining neighbours' components in a second gives
    eq. (complex_step) (Section 2)."""
    u = inputs.random_words(14, 11, seed=8)[0]
    ref = oracle_lib.wide2(u, 5)
    v = u.copy()
    with np.errstate(over="ignore"):
        for _ in range(5):
            # sub-step 1: component k of the 5-vector (x along axis 1)
            half = np.stack([v, np.roll(v, 1, axis=1), np.roll(v, -1, axis=1),
                             np.roll(v, 1, axis=0), np.roll(v, -1, axis=0)])
            # sub-step 2: west neighbour's 2nd, east's 3rd, north's 4th, south's 5th
            v = (np.roll(half[1], 1, axis=1) + np.roll(half[2], -1, axis=1)
                 + np.roll(half[3], 1, axis=0) + np.roll(half[4], -1, axis=0)
                 - np.uint64(4) * half[0])
    assert np.array_equal(v, ref)


# ------------------------------------------------------------------------- euler

GAMMA, CFL, KAPPA = 1.4, 0.3, 0.5


def _euler_state(rho, m, q, p):
    E = p / (GAMMA - 1.0) + 0.5 * (m * m + q * q) / rho
    return np.stack([rho, m, q, E]).astype(np.float64)


def test_euler_wavespeed_and_dt_closed_form(oracle_lib):
    """Uniform gas at rest with p = rho = 1: a = sqrt(gamma); moving with
    u = 0.5: a = 0.5 + sqrt(gamma); dt = cfl min(dx, dy) / a."""
    ny, nx = 6, 8
    one = np.ones((ny, nx))
    a, dt = oracle_lib.euler_setup(_euler_state(one, 0 * one, 0 * one, one), GAMMA, CFL)
    assert a == pytest.approx(np.sqrt(GAMMA), rel=4 * EPS)
    assert dt == pytest.approx(CFL * (1.0 / nx) / np.sqrt(GAMMA), rel=8 * EPS)
    a2, _ = oracle_lib.euler_setup(_euler_state(one, 0.5 * one, 0 * one, one), GAMMA, CFL)
    assert a2 == pytest.approx(0.5 + np.sqrt(GAMMA), rel=8 * EPS)


def test_euler_free_stream_is_preserved_bitwise(oracle_lib):
    ny, nx = 8, 12
    one = np.ones((ny, nx))
    U0 = _euler_state(1.2 * one, 0.3 * one, -0.1 * one, 0.9 * one)
    a, dt = oracle_lib.euler_setup(U0, GAMMA, CFL)
    UT = oracle_lib.euler_rk2(U0, GAMMA, dt, KAPPA, a, 25)
    assert np.array_equal(UT, U0)


def test_euler_gas_at_rest_with_uniform_pressure(oracle_lib):
    """rho = 1 + 0.1 cos(theta x), u = v = 0, p = 1: the fluxes F, G are uniform,
    so m and q stay exactly 0 and E exactly constant, and rho follows the
    dissipation alone -- a linear scheme whose Fourier factor per midpoint RK2
    step is G = 1 + z + z^2/2, z = dt kax (2 cos theta - 2)."""
    ny, nx, k = 6, 32, 2
    x = np.arange(nx)
    theta = 2 * np.pi * k / nx
    rho = np.tile(1.0 + 0.1 * np.cos(theta * x), (ny, 1))
    U0 = _euler_state(rho, 0 * rho, 0 * rho, np.ones_like(rho))
    a, dt = oracle_lib.euler_setup(U0, GAMMA, CFL)
    T = 60
    UT = oracle_lib.euler_rk2(U0, GAMMA, dt, KAPPA, a, T)
    assert np.all(UT[1] == 0.0) and np.all(UT[2] == 0.0)
    assert np.array_equal(UT[3], U0[3])
    kax = KAPPA * a * nx
    z = dt * kax * (2 * np.cos(theta) - 2)
    G = 1 + z + z * z / 2
    assert abs(G) < 1.0
    pred = 1.0 + 0.1 * G ** T * np.cos(theta * x)
    assert np.max(np.abs(UT[0] - pred[None, :])) < 1e-13


def test_euler_linear_acoustics(oracle_lib):
    """A small perturbation of a gas at rest (rho0 = p0 = 1) follows the
    linearised scheme: fluxes F ~ A w with A = [[0,1,0],[0,0,g-1],[0,g/(g-1),0]]
    on w = (rho', m', E'), so per step w^ <- (I + Z + Z^2/2) w^ with
    Z = dt (kax (2 cos th - 2) I - 2 i cx sin th A). Catches any error in the
    pressure, the momentum flux or the energy flux."""
    ny, nx, k, delta, T = 4, 32, 3, 1e-6, 40
    x = np.arange(nx)
    theta = 2 * np.pi * k / nx
    w_hat = np.array([0.7, -0.4, 1.3])
    c = np.cos(theta * x)
    rho = np.tile(1.0 + delta * w_hat[0] * c, (ny, 1))
    m = np.tile(delta * w_hat[1] * c, (ny, 1))
    E = np.tile(1.0 / (GAMMA - 1.0) + delta * w_hat[2] * c, (ny, 1))
    U0 = np.stack([rho, m, np.zeros_like(rho), E])
    a, dt = oracle_lib.euler_setup(U0, GAMMA, CFL)
    UT = oracle_lib.euler_rk2(U0, GAMMA, dt, KAPPA, a, T)
    A = np.array([[0, 1, 0], [0, 0, GAMMA - 1], [0, GAMMA / (GAMMA - 1), 0]], dtype=complex)
    cx, kax = 0.5 * nx, KAPPA * a * nx
    Z = dt * (kax * (2 * np.cos(theta) - 2) * np.eye(3) - 2j * cx * np.sin(theta) * A)
    G = np.eye(3) + Z + Z @ Z / 2
    wT = np.linalg.matrix_power(G, T) @ w_hat
    pred = np.real(wT[:, None] * np.exp(1j * theta * x)[None, :])      # (3, nx)
    got = np.stack([UT[0, 0] - 1.0, UT[1, 0], UT[3, 0] - 1.0 / (GAMMA - 1.0)]) / delta
    assert np.max(np.abs(got - pred)) < 1e-4
    assert np.all(UT[2] == 0.0)
    # and the perturbation really moved (it is not the identity map)
    assert np.max(np.abs(pred - w_hat[:, None] * c[None, :])) > 0.1


def test_euler_conserves_all_four_sums(oracle_lib):
    U0 = inputs.euler_pulse(24, 20, seed=2)
    a, dt = oracle_lib.euler_setup(U0, GAMMA, CFL)
    UT = oracle_lib.euler_rk2(U0, GAMMA, dt, KAPPA, a, 50)
    for c in range(4):
        scale = np.sum(np.abs(U0[c])) + 1.0
        assert abs(UT[c].sum() - U0[c].sum()) <= 1e-12 * scale
    assert np.max(np.abs(UT[1])) > 1e-4      # the pulse set the gas moving


def test_euler_transpose_symmetry_on_square_grids(oracle_lib):
    """Swapping x with y (and m with q) maps the scheme to itself. The fused
    multiply-adds round the two axes' terms in a fixed order, so the images agree
    to rounding (any swapped index or axis constant would show at O(1e-3))."""
    U0 = inputs.euler_pulse(16, 16, seed=9)
    a, dt = oracle_lib.euler_setup(U0, GAMMA, CFL)
    UT = oracle_lib.euler_rk2(U0, GAMMA, dt, KAPPA, a, 12)
    Ut0 = np.stack([U0[0].T, U0[2].T, U0[1].T, U0[3].T])
    UtT = oracle_lib.euler_rk2(Ut0, GAMMA, dt, KAPPA, a, 12)
    mirror = np.stack([UT[0].T, UT[2].T, UT[1].T, UT[3].T])
    assert np.max(np.abs(UtT - mirror)) <= 1e-13
    assert np.max(np.abs(UT - U0)) > 1e-4


# ------------------------------------------------------- reduced-precision heat

def test_bf16_rounding_is_round_to_nearest_even(oracle_lib):
    """Hand-checked ties and a library conversion (torch's float32 -> bfloat16,
    round to nearest even) on random values across many binades."""
    assert oracle_lib.f32_to_bf16(1.0) == 0x3F80
    assert oracle_lib.f32_to_bf16(1.0 + 2 ** -8) == 0x3F80          # tie -> even
    assert oracle_lib.f32_to_bf16(1.0 + 3 * 2 ** -8) == 0x3F82      # tie -> even
    assert oracle_lib.f32_to_bf16(1.0 + 2 ** -8 + 2 ** -20) == 0x3F81
    assert oracle_lib.f32_to_bf16(-2.0) == 0xC000
    assert oracle_lib.bf16_to_f32(0x3F81) == 1.0078125
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    x = (rng.standard_normal(2000) * 10.0 ** rng.uniform(-20, 20, 2000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    got = np.array([oracle_lib.f32_to_bf16(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, ref)


def _plain_f32_heat(u0, r, T):
    """Uncompensated binary32 forward Euler (numpy), the baseline Kahan improves on."""
    u = u0.astype(np.float32)
    r = np.float32(r)
    for _ in range(T):
        s = (np.roll(u, -1, 1) + np.roll(u, -1, 0)) + (np.roll(u, 1, 1) + np.roll(u, 1, 0))
        u = u + r * (s - np.float32(4) * u)
    return u


def test_heat_kahan_f32_tracks_fp64_better_than_plain_f32(oracle_lib):
    """A slowly decaying mode (per-step increments ~1e-3 of u): the compensated
    accumulation keeps the binary32 result closer to the FP64 one than
    uncompensated binary32 arithmetic (the stencil still reads the rounded
    stored values, which bounds the gain to a few times), and it still follows
    the exact decay."""
    n, T = 64, 2000
    u64 = 1.0 + 0.5 * inputs.fourier_mode(n, n, 1, 1)
    ref = oracle_lib.heat(u64, 0.2, T)
    u, c = oracle_lib.heat_kahan(u64.astype(np.float32), np.zeros((n, n), np.float32), 0.2, T)
    err_kahan = np.max(np.abs(u.astype(np.float64) - ref))
    err_plain = np.max(np.abs(_plain_f32_heat(u64, 0.2, T).astype(np.float64) - ref))
    assert err_kahan < err_plain / 2.5
    assert err_kahan < 1e-6
    g = 1.0 - 0.8 * (2 * np.sin(np.pi / n) ** 2)
    assert np.max(np.abs(u - (1.0 + 0.5 * g ** T * inputs.fourier_mode(n, n, 1, 1)))) < 2e-6


def test_heat_kahan_zero_rate_and_compensation_identity(oracle_lib):
    """r = 0 with no pending compensation leaves u and c unchanged; with r > 0
    the stored pair satisfies the compensated-sum identities u' = u + y and
    c' = (u' - u) - y at every point, y = delta - c, with the increment
    recomputed in float32 by numpy."""
    rng = np.random.default_rng(4)
    u0 = rng.random((12, 10)).astype(np.float32)
    c0 = (rng.standard_normal((12, 10)) * 1e-8).astype(np.float32)
    u, c = oracle_lib.heat_kahan(u0, np.zeros_like(u0), 0.0, 5)
    assert np.array_equal(u, u0) and np.all(c == 0)
    u1, c1 = oracle_lib.heat_kahan(u0, c0, 0.2, 1)
    f = np.float32
    s = (np.roll(u0, -1, 1) + np.roll(u0, -1, 0)) + (np.roll(u0, 1, 1) + np.roll(u0, 1, 0))
    d = (s.astype(np.float64) - 4.0 * u0.astype(np.float64)).astype(np.float32)   # fused: one rounding
    y = f(0.2) * d - c0
    assert np.array_equal(u1, u0 + y)
    assert np.array_equal(c1, (u1 - u0) - y)


def test_heat_kahan_bf16_storage_keeps_small_increments(oracle_lib):
    """With bfloat16 storage (8-bit significand) the per-step increments of a
    slow mode fall below half an ulp of u: uncompensated (numpy float32 update,
    rounded to bfloat16 by the oracle's rounding) the field stagnates; with the
    compensation it keeps following the FP64 solution to within a few times the
    error of representing the initial field in bfloat16."""
    n, T = 32, 300
    x = np.arange(n)
    u64 = np.tile(1.0 + 0.25 * np.cos(2 * np.pi * x / n), (n, 1))
    ref = oracle_lib.heat(u64, 0.2, T)
    bits = np.vectorize(lambda v: oracle_lib.f32_to_bf16(float(v)), otypes=[np.uint16])
    tofl = np.vectorize(oracle_lib.bf16_to_f32, otypes=[np.float64])
    u0 = bits(u64.astype(np.float32))
    rep_err = np.max(np.abs(tofl(u0) - u64))
    u, c = oracle_lib.heat_kahan(u0, np.zeros_like(u0), 0.2, T, storage="bf16")
    err_kahan = np.max(np.abs(tofl(u) - ref))
    plain = tofl(u0)
    for _ in range(T):
        s = (np.roll(plain, -1, 1) + np.roll(plain, -1, 0)) + (np.roll(plain, 1, 1) + np.roll(plain, 1, 0))
        plain = tofl(bits((plain + 0.2 * (s - 4 * plain)).astype(np.float32)))
    err_plain = np.max(np.abs(plain - ref))
    assert np.max(np.abs(ref - 1.0)) < 0.25 * 0.2          # the mode really decayed
    assert err_kahan < 3 * rep_err
    assert err_plain > 10 * err_kahan


# --------------------------------------------------- Euler, precision forms

EPS32 = float(np.finfo(np.float32).eps)


def _ek_state(U, storage, oracle_lib):
    """(U, U*, C) with U* = U and C = 0, U rounded to the storage format;
    returns (state, U as float64)."""
    U32 = np.asarray(U, dtype=np.float32)
    if storage == "bf16":
        bits = np.vectorize(lambda v: oracle_lib.f32_to_bf16(float(v)), otypes=[np.uint16])(U32)
        U32 = oracle_lib.bf16_bits_to_f32(bits)
    S = np.concatenate([U32, U32, np.zeros_like(U32)])
    if storage == "bf16":
        S = oracle_lib.f32_to_bf16_bits(S)
    return S, U32.astype(np.float64)


def _ek_values(S, storage, oracle_lib):
    return (oracle_lib.bf16_bits_to_f32(S) if storage == "bf16" else S).astype(np.float64)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_euler_kahan_free_stream_and_gas_at_rest_are_exact(oracle_lib, storage):
    """A uniform moving state is a fixed point bit for bit (every difference
    is 0, so the increments and the compensation stay 0); a gas at rest with
    uniform pressure keeps m = q = 0 and E exactly, whatever the storage."""
    ny, nx = 8, 12
    one = np.ones((ny, nx))
    U0 = _euler_state(1.25 * one, 0.375 * one, -0.125 * one, 0.875 * one)
    S, Uf = _ek_state(U0, storage, oracle_lib)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    assert np.array_equal(oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, 20, storage), S)
    x = np.arange(32)
    rho = np.tile(1.0 + 0.1 * np.cos(2 * np.pi * 2 * x / 32), (6, 1))
    S, Uf = _ek_state(_euler_state(rho, 0 * rho, 0 * rho, np.ones_like(rho)), storage, oracle_lib)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    V = _ek_values(oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, 40, storage), storage, oracle_lib)
    assert np.all(V[1] == 0) and np.all(V[2] == 0) and np.all(V[5] == 0) and np.all(V[6] == 0)
    assert np.array_equal(V[3], Uf[3]) and np.all(V[11] == 0)
    assert np.max(np.abs(V[0] - 1.0)) < 0.1          # rho diffuses towards its mean


@pytest.mark.parametrize("T", [100, 1000])
def test_euler_kahan_f32_tracks_the_fp64_scheme(oracle_lib, T):
    """From the same (binary32) initial pressure pulse, the binary32 form stays
    within a few binary32 roundings (8 eps32 of max |U|) of the FP64 oracle,
    far below each variable's own change over the first 100 steps: a dropped
    term, a wrong sign or a swapped flux would leave errors of that size."""
    n = 32
    S, Uf = _ek_state(inputs.euler_pulse(n, n, 2, gamma=GAMMA), "f32", oracle_lib)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    ref = oracle_lib.euler_rk2(Uf, GAMMA, dt, KAPPA, a, T)
    V = _ek_values(oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, T, "f32"), "f32", oracle_lib)
    err = np.max(np.abs(V[:4] - ref), axis=(1, 2))
    change = np.max(np.abs(ref - Uf), axis=(1, 2))
    assert np.all(err <= 8 * EPS32 * np.max(np.abs(ref)))
    if T == 100:          # later the momentum of the pulse has decayed to ~1e-9
        assert np.all(err <= 0.01 * change)


def test_euler_kahan_bf16_compensation_keeps_the_small_increments(oracle_lib):
    """bfloat16 storage (8-bit significand): the per-step increments of the
    decaying pulse fall below half an ulp of U. With the compensation reset
    before every step (the same oracle, one step at a time: plain rounding) the
    field stagnates far from the FP64 solution; compensated it stays within
    half a bfloat16 ulp of max |U| and 20x closer, and the compensated sums
    sum(U - C) drift 10x less than the stored sums sum(U)."""
    n, T = 32, 1000
    S, Uf = _ek_state(inputs.euler_pulse(n, n, 2, gamma=GAMMA), "bf16", oracle_lib)
    a, dt = oracle_lib.euler_setup(Uf, GAMMA, CFL)
    ref = oracle_lib.euler_rk2(Uf, GAMMA, dt, KAPPA, a, T)
    K = _ek_values(oracle_lib.euler_kahan(S, GAMMA, dt, KAPPA, a, T, "bf16"), "bf16", oracle_lib)
    P = S.copy()
    for _ in range(T):
        P = oracle_lib.euler_kahan(P, GAMMA, dt, KAPPA, a, 1, "bf16")
        P[8:] = 0
    P = _ek_values(P, "bf16", oracle_lib)
    err_k = np.max(np.abs(K[:4] - ref))
    err_p = np.max(np.abs(P[:4] - ref))
    half_ulp = 2.0 ** np.floor(np.log2(np.max(np.abs(ref)))) * 2.0 ** -8
    assert err_k < half_ulp
    assert err_p > 20 * err_k
    s0 = Uf.sum(axis=(1, 2))
    drift_comp = np.abs((K[:4] - K[8:]).sum(axis=(1, 2)) - s0)
    drift_stored = np.abs(K[:4].sum(axis=(1, 2)) - s0)
    assert drift_comp[0] * 10 < drift_stored[0] and drift_comp[3] * 10 < drift_stored[3]


# ------------------------------------------------------------------------ wave

@pytest.mark.parametrize("T", [50, 400])
def test_wave_single_mode_oscillates_with_the_leapfrog_frequency(oracle_lib, T):
    """For a mode with discrete Laplacian eigenvalue lam, the leapfrog recurrence
    u^{n+1} = (2 + C^2 lam) u^n - u^{n-1} has u^n = cos(n th) mode with
    cos th = 1 + C^2 lam / 2 when u^{-1} = cos(th) mode (Section 6's CFL 0.3)."""
    n, p, q, C2 = 32, 2, 3, 0.3 ** 2
    mode = inputs.fourier_mode(n, n, p, q)
    lam = -4 * (np.sin(np.pi * p / n) ** 2 + np.sin(np.pi * q / n) ** 2)
    th = np.arccos(1 + C2 * lam / 2)
    u, uo = oracle_lib.wave(mode, np.cos(th) * mode, C2, T)
    assert np.max(np.abs(u - np.cos(T * th) * mode)) < 4 * T * EPS * 4
    assert np.max(np.abs(uo - np.cos((T - 1) * th) * mode)) < 4 * T * EPS * 4


def test_wave_impulse_response_and_mean_velocity(oracle_lib):
    """One step from a unit impulse at rest: 2 - 1 - 4C^2 at the centre, C^2 at
    the 4 edge neighbours; over many steps the mean velocity sum(u^n - u^{n-1})
    is conserved (the Laplacian sums to zero on the periodic grid)."""
    C2 = 0.09
    u0 = np.zeros((9, 11))
    u0[4, 5] = 1.0
    u1, uo1 = oracle_lib.wave(u0, u0, C2, 1)
    expect = np.zeros_like(u0)
    expect[4, 5] = 1.0 - 4.0 * C2      # 4 C^2 is exact: one rounding, as in the fused form
    for dj, di in [(0, 1), (0, -1), (1, 0), (-1, 0)]:
        expect[4 + dj, 5 + di] = C2
    assert np.allclose(u1, expect, rtol=0, atol=1e-16) and np.array_equal(uo1, u0)
    rng = np.random.default_rng(3)
    a, b = rng.random((20, 24)), rng.random((20, 24))
    v0 = np.sum(a - b)
    u, uo = oracle_lib.wave(a, b, C2, 300)
    assert abs(np.sum(u - uo) - v0) < 1e-10
