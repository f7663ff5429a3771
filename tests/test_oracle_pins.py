"""Pins of the FP64 oracle against closed forms, invariants and independent routines.

Each test fixes one stage of the oracle to something other than itself, so that a dropped
term, a sign or index error or a transposed operand in that stage fails here:

* FFT: numpy.fft (independent implementation), all radices used (2, 5 and others).
* Spot: exact discrete Dirichlet form of a flat square subaperture; Parseval; an integer tilt
  rolls the image exactly; elongation equals circular convolution with the periodised
  Gaussian (Poisson summation) along the stated direction.
* Binning and centroid: hand-built images with known answers.
* Bilinear sampling: exact on affine screens (asymmetric coefficients catch transposition).
* Cone projection: a linear layer seen by a laser star at finite height gives
  b.(x (1 - h/H) + h theta + t v) exactly.
* DM: single poke equals the Gaussian closed form with g(pitch) = coupling; the separable
  evaluation equals the brute-force double sum on a non-square actuator grid.
* Science: zero residual gives Strehl 1 and a unit PSF peak; Parseval of the PSF; Marechal
  regime exp(-sigma^2) for a small random phase.
* Integrator: with a static DM-shaped aberration and R = -pinv(D), the command error decays as
  (1 - g)^k.
* Noise: Poisson and read-noise moments; float exp/log/cos against libm.
* Screens: structure function against the quadrature of the von Karman spectrum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n", [1, 2, 7, 14, 16, 32, 64, 243, 256, 1000, 1280])
def test_fft1_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    assert np.max(np.abs(oracle.fft1(x) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(oracle.fft1(x, inverse=True) - np.fft.ifft(x))) <= 1e-13 * max(1.0, n)


@pytest.mark.parametrize("n", [8, 16, 32, 64, 40])
def test_fft2_matches_numpy(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ref = np.fft.fft2(x)
    assert np.max(np.abs(oracle.fft2(x) - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(oracle.fft2(x, inverse=True) - np.fft.ifft2(x))) <= 1e-13 * n


# ------------------------------------------------------------------------------------------ spot
def _dirichlet(kp, n, N):
    return (np.sin(np.pi * kp * n / N) / np.sin(np.pi * kp / N)) ** 2


@pytest.mark.parametrize("n,N", [(8, 16), (8, 32), (32, 64), (5, 20)])
def test_flat_spot_is_dirichlet(n, N):
    img = oracle.sh_image(np.ones((n, n)), np.zeros((n, n)), N)
    kp = (np.arange(N) - N / 2) + 0.5          # half-bin centring: peak at N/2 - 1/2
    d = _dirichlet(kp, n, N)
    ref = np.outer(d, d)
    assert np.max(np.abs(img - ref)) <= 1e-10 * ref.max()
    assert img.sum() == pytest.approx(N * N * n * n, rel=1e-12)


@pytest.mark.parametrize("sigma", [0.0, 1.7])
def test_spot_parseval(sigma):
    rng = np.random.default_rng(5)
    n, N = 8, 32
    amp = (rng.random((n, n)) > 0.2).astype(float)
    ph = rng.standard_normal((n, n)) * 2.0
    img = oracle.sh_image(amp, ph, N, sigma, (0.6, 0.8))
    assert abs(img.sum() - N * N * (amp ** 2).sum()) <= 1e-10 * img.sum()


@pytest.mark.parametrize("m,axis", [(3, 1), (-5, 1), (2, 0), (-1, 0)])
def test_integer_tilt_rolls_spot(m, axis):
    rng = np.random.default_rng(9)
    n, N = 8, 32
    amp = (rng.random((n, n)) > 0.1).astype(float)
    base = rng.standard_normal((n, n)) * 0.7
    y, x = np.mgrid[0:n, 0:n]
    ramp = 2 * np.pi * m * (x if axis == 1 else y) / N
    i0 = oracle.sh_image(amp, base, N)
    i1 = oracle.sh_image(amp, base + ramp, N)
    assert np.max(np.abs(i1 - np.roll(i0, m, axis=axis))) <= 1e-10 * i0.max()


def _periodised_gaussian(N, sigma):
    j = np.arange(N)
    k = np.zeros(N)
    for p in range(-6, 7):
        t = j - p * N
        k += np.exp(-t * t / (2 * sigma * sigma))
    return k / (math.sqrt(2 * math.pi) * sigma)


@pytest.mark.parametrize("direction,axis", [((1.0, 0.0), 1), ((0.0, 1.0), 0), ((-1.0, 0.0), 1)])
def test_elongation_is_periodic_gaussian_convolution(direction, axis):
    n, N, sigma = 8, 32, 2.5
    rng = np.random.default_rng(3)
    amp = np.ones((n, n))
    ph = rng.standard_normal((n, n)) * 0.5
    plain = oracle.sh_image(amp, ph, N)
    elong = oracle.sh_image(amp, ph, N, sigma, direction)
    K = _periodised_gaussian(N, sigma)
    # circular convolution along the elongation axis
    ref = np.zeros_like(plain)
    for s in range(N):
        ref += K[s] * np.roll(plain, s, axis=axis)
    assert np.max(np.abs(elong - ref)) <= 1e-8 * plain.max()


def test_elongation_direction_symmetry():
    n, N, sigma = 8, 32, 3.0
    flat = np.zeros((n, n))
    amp = np.ones((n, n))
    d = 1 / math.sqrt(2)
    a = oracle.sh_image(amp, flat, N, sigma, (d, d))
    b = oracle.sh_image(amp, flat, N, sigma, (d, -d))
    assert np.max(np.abs(a - a.T)) <= 1e-9 * a.max()
    # mirror x -> N-1-x maps the (1,1) streak onto the (1,-1) streak (flat spot centre N/2-1/2)
    assert np.max(np.abs(b - a[:, ::-1])) <= 1e-9 * a.max()
    assert not np.allclose(a, b, rtol=1e-3)


def test_binning_and_cog():
    img = np.arange(64.0).reshape(8, 8)
    out = oracle.bin_image(img, 2)
    ref = img.reshape(4, 2, 4, 2).sum(axis=(1, 3))
    assert np.array_equal(out, ref)
    d = np.zeros((16, 16))
    d[3, 12] = 5.0
    sx, sy = oracle.cog(d)
    assert sx == pytest.approx(12 - 7.5) and sy == pytest.approx(3 - 7.5)
    assert oracle.cog(np.zeros((8, 8))) == (0.0, 0.0)
    e = np.zeros((8, 8))
    e[2, 2] = 1.0
    e[2, 5] = 3.0
    sx, sy = oracle.cog(e)
    assert sx == pytest.approx((1.0 * (2 - 3.5) + 3.0 * (5 - 3.5)) / 4.0)
    assert sy == pytest.approx(2 - 3.5)


def test_cog_antisymmetric_and_linear_in_small_tilt():
    n, N, b = 8, 32, 2
    amp = np.ones((n, n))
    x = np.mgrid[0:n, 0:n][1]
    res = []
    for a in (-0.2, -0.1, 0.1, 0.2):  # tilt in FFT bins
        img = oracle.bin_image(oracle.sh_image(amp, 2 * np.pi * a * x / N, N), b)
        res.append(oracle.cog(img)[0])
    assert res[0] == pytest.approx(-res[3], abs=1e-12)
    assert res[1] == pytest.approx(-res[2], abs=1e-12)
    # gain close to 1/b detector pixel per FFT bin, linear in the tilt
    assert res[3] / 0.2 == pytest.approx(1.0 / b, rel=0.15)
    assert res[3] / res[2] == pytest.approx(2.0, rel=0.01)


# ------------------------------------------------------------------------------------------ geometry
def test_bilinear_affine_exact_and_periodic():
    n = 40
    y, x = np.mgrid[0:n, 0:n].astype(float)
    s = 0.3 + 1.7 * x - 0.9 * y
    rng = np.random.default_rng(2)
    for _ in range(50):
        fx, fy = rng.uniform(0, n - 1.001, 2)
        assert oracle.bilinear_periodic(s, fx, fy) == pytest.approx(0.3 + 1.7 * fx - 0.9 * fy, abs=1e-11)
    r = rng.standard_normal((n, n))
    assert oracle.bilinear_periodic(r, 5.0, 7.0) == r[7, 5]
    assert oracle.bilinear_periodic(r, n - 0.5, 3.0) == pytest.approx(0.5 * (r[3, n - 1] + r[3, 0]))
    assert oracle.bilinear_periodic(r, -1.0, -2.0) == r[n - 2, n - 1]


def test_bilinear_clamped_affine_edges_and_library():
    """The DM sampling rule: exact on an affine grid at fractional indices (unequal x and y
    coefficients, so a transposed index fails), the edge value beyond both edges, the last cell
    capped at n - 2, and equal everywhere to scipy's order-1 map_coordinates with nearest-edge
    extension, an independent implementation of clamped bilinear interpolation."""
    from scipy import ndimage
    n = 23
    y, x = np.mgrid[0:n, 0:n].astype(float)
    s = 0.3 + 1.7 * x - 0.9 * y
    rng = np.random.default_rng(12)
    for fx, fy in rng.uniform(0.0, n - 1.0, (60, 2)):
        assert oracle.bilinear_clamped(s, fx, fy) == pytest.approx(0.3 + 1.7 * fx - 0.9 * fy, abs=1e-12)
    r = rng.standard_normal((n, n))
    pts = [tuple(p) for p in rng.uniform(-3.0, n + 2.0, (200, 2))]
    pts += [(0.0, 0.0), (n - 1.0, n - 1.0), (n - 1.0, 4.5), (4.5, n - 1.0), (n - 1.5, n - 1.25),
            (-0.5, 6.3), (n - 0.2, 6.3), (6.3, -7.0), (6.3, n + 9.0), (-2.0, n + 2.0), (9.0, 11.0)]
    for fx, fy in pts:
        ref = ndimage.map_coordinates(r, [[fy], [fx]], order=1, mode="nearest")[0]
        assert oracle.bilinear_clamped(r, fx, fy) == pytest.approx(ref, abs=1e-13), (fx, fy)
    assert oracle.bilinear_clamped(r, -4.2, 7.0) == r[7, 0]
    assert oracle.bilinear_clamped(r, n + 3.5, 7.0) == r[7, n - 1]
    assert oracle.bilinear_clamped(r, 5.0, -1.0) == r[0, 5]
    assert oracle.bilinear_clamped(r, 5.0, n + 1.0) == r[n - 1, 5]
    assert oracle.bilinear_clamped(r, n - 1.0, n - 1.0) == r[n - 1, n - 1]
    assert oracle.bilinear_clamped(r, n - 1.75, 3.0) == pytest.approx(0.75 * r[3, n - 2] + 0.25 * r[3, n - 1],
                                                                       abs=1e-14)
    assert oracle.bilinear_clamped(r, 9.0, 11.0) == r[11, 9]
    # the right edge stays in the last cell (columns n-2, n-1): a sample outside it, here the
    # first sample of the next row, must not enter the sum even with a zero weight
    r2 = r.copy()
    r2[5, 0] = np.inf
    assert oracle.bilinear_clamped(r2, n - 1.0, 4.0) == r2[4, n - 1]
    assert oracle.bilinear_clamped(r2, n + 2.0, 4.0) == r2[4, n - 1]


def _poked_altitude_dm_case(frac_x, frac_y, surf_n):
    """One laser star at 90 km and one DM at 5 km whose surface pitch is the cone-compressed
    pupil pitch; the star's direction moves the footprint by (3 + frac_x, -2 + frac_y) surface
    samples.  Actuator (row 3, column 7) of an 11 x 11 grid is poked to 1.3 rad."""
    h, H, D = 5000.0, 90e3, 4.0
    N = 4 * 8
    dx = D / N
    f = 1.0 - h / H
    sdx = dx * f
    theta = ((3.0 + frac_x) * sdx / h, (-2.0 + frac_y) * sdx / h)
    cfg = _small_cfg(alt=0.0, kind="lgs", theta=theta)
    nx, pitch, coup = 11, 0.5, 0.3
    cfg["dms"] = [{"alt": h, "pitch": pitch, "coupling": coup, "nx": nx, "ny": nx,
                   "valid": np.ones((nx, nx), np.uint8), "surf_n": surf_n, "surf_dx": sdx}]
    sim = oracle.Sim(cfg, [np.zeros((256, 256), np.float32)])
    c = np.zeros(sim.n_cmd)
    c[3 * nx + 7] = 1.3
    sim.set_commands(c)
    X = (np.arange(N) - 0.5 * (N - 1)) * dx
    u = X[None, :] * f + h * theta[0] + 0.0 * X[:, None]
    v = X[:, None] * f + h * theta[1] + 0.0 * X[None, :]
    return sim, u, v, sdx, (nx, pitch, coup)


def test_dm_at_altitude_on_grid_is_gaussian_closed_form():
    """Every pupil sample of the laser star projects onto a surface sample of the 5 km DM
    (whole-sample offset), so the residual phase must be minus the Gaussian poke evaluated at
    the cone-beam point x (1 - h/H) + h theta: a closed form through the projection and the
    clamped sampler with no interpolation."""
    sim, u, v, _, (nx, pitch, coup) = _poked_altitude_dm_case(0.0, 0.0, 48)
    ph = sim.wfs_phase(0)
    sig = pitch / math.sqrt(2.0 * math.log(1.0 / coup))
    xa, yb = (7 - 0.5 * (nx - 1)) * pitch, (3 - 0.5 * (nx - 1)) * pitch
    ref = -1.3 * np.exp(-((u - xa) ** 2 + (v - yb) ** 2) / (2.0 * sig * sig))
    assert np.max(np.abs(ph - ref)) < 1e-12
    assert ph.min() < -0.5


def test_dm_at_altitude_fractional_and_off_grid():
    """A fractional footprint offset, with part of the footprint beyond the surface grid on two
    sides: the residual phase equals minus scipy's clamped bilinear interpolation of the surface
    at the projected indices u / dx + (n - 1) / 2."""
    from scipy import ndimage
    surf_n = 30
    sim, u, v, sdx, _ = _poked_altitude_dm_case(0.37, -0.21, surf_n)
    ph = sim.wfs_phase(0)
    S = sim.dm_surface(0)
    fx = u / sdx + 0.5 * (surf_n - 1)
    fy = v / sdx + 0.5 * (surf_n - 1)
    assert fx.max() > surf_n - 1 and fy.min() < 0.0          # the footprint leaves the grid
    ref = -ndimage.map_coordinates(S, [fy.ravel(), fx.ravel()], order=1, mode="nearest").reshape(ph.shape)
    assert np.max(np.abs(ph - ref)) < 1e-12
    assert np.max(np.abs(ph)) > 0.1


def test_flux_is_photons_times_illuminated_fraction():
    """Noise-free detector frames sum to n_photons times the subaperture's illuminated fraction
    (flux reading), the fraction counted here by brute force over the annular pupil samples.
    Covers partially illuminated subapertures, an elongated laser spot and a natural star."""
    D, obs, nsub, npx = 4.0, 0.3, 8, 8
    cfg = _small_cfg(alt=0.0, kind="lgs")
    cfg["obstruction"] = obs
    cfg["wfs"] = [inputs._wfs("lgs", (6 * inputs.ARCSEC, 0.0), nsub, npx, 16, 2, 589e-9, 750.0, height=90e3,
                              na_fwhm=10e3, launch=(1.1, -0.4)),
                  inputs._wfs("ngs", (0.0, 3 * inputs.ARCSEC), nsub, npx, 16, 1, 500e-9, 320.0)]
    scr = inputs.phase_screen(256, 0.125, 0.2, 25.0, 5)
    sim = oracle.Sim(cfg, [scr])
    sim.measure()
    n = nsub * npx
    partial = 0
    for w, ww in enumerate(cfg["wfs"]):
        lam, _ = sim.frames(w)
        for q, idx in enumerate(sim.valid(w)):
            sy, sx = divmod(int(idx), nsub)
            yy = (sy * npx + np.arange(npx)[:, None] - 0.5 * (n - 1)) * (D / n)
            xx = (sx * npx + np.arange(npx)[None, :] - 0.5 * (n - 1)) * (D / n)
            r2 = xx * xx + yy * yy
            frac = np.sum((r2 <= (D / 2) ** 2) & (r2 >= (obs * D / 2) ** 2)) / float(npx * npx)
            partial += frac < 1.0
            expect = ww["n_photons"] * frac
            assert abs(float(lam[q].sum(dtype=np.float64)) - expect) <= 1e-6 * expect, (w, q)
    assert partial >= 8


def test_valid_subaps_brute_force():
    for D, obs, ns, npx, expect in [(8.0, 0.0, 16, 8, None), (39.0, 0.28, 80, 8, None), (39.0, 0.28, 2, 32, 4)]:
        A = oracle.pupil(D, obs, ns * npx)
        n = ns * npx
        cnt = 0
        for sy in range(ns):
            for sx in range(ns):
                inside = 0
                for yy in range(npx):
                    yv = (sy * npx + yy - 0.5 * (n - 1)) * (D / n)
                    xv = (sx * npx + np.arange(npx) - 0.5 * (n - 1)) * (D / n)
                    r2 = xv * xv + yv * yv
                    inside += int(np.sum((r2 <= (D / 2) ** 2) & (r2 >= (obs * D / 2) ** 2)))
                cnt += inside * 2 >= npx * npx
        c2, vmap, _ = oracle.valid_subaps(A, ns, npx, 0.5)
        assert c2 == cnt
        assert np.array_equal(vmap, vmap[::-1, :]) and np.array_equal(vmap, vmap.T)
        if expect is not None:
            assert c2 == expect


def _small_cfg(alt=5000.0, kind="lgs", theta=(10 * inputs.ARCSEC, -5 * inputs.ARCSEC)):
    cfg = {
        "name": "probe", "D": 4.0, "obstruction": 0.0, "lambda_ref": 500e-9, "dt": 0.01, "gain": 0.5,
        "seed": 3, "noise": False, "psf_every": 1,
        "wfs": [inputs._wfs(kind, theta, 4, 8, 16, 2, 600e-9, 100.0, height=90e3 if kind == "lgs" else 0.0)],
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 32, "pad": 2}],
        "layers": [{"n": 256, "pixel": 0.125, "alt": alt, "vx": 2.0, "vy": -1.0, "r0": 0.2, "L0": 25.0, "seed": 1}],
    }
    cfg["dms"] = [inputs.dm_spec(cfg, 0.0, 0.5, 0.3, nx=9)]
    return cfg


@pytest.mark.parametrize("kind", ["lgs", "ngs"])
def test_cone_projection_of_linear_layer(kind):
    cfg = _small_cfg(kind=kind)
    n = 256
    X = (np.arange(n) - 0.5 * (n - 1)) * 0.125
    bx, by = 0.37, -0.21
    scr = (bx * X[None, :] + by * X[:, None]).astype(np.float32)
    sim = oracle.Sim(cfg, [scr])
    sim.k = 3
    ph = sim.wfs_phase(0)
    N = 32
    x = (np.arange(N) - 0.5 * (N - 1)) * (4.0 / N)
    h, H = 5000.0, 90e3
    f = 1 - h / H if kind == "lgs" else 1.0
    th = cfg["wfs"][0]["theta"]
    t = 3 * 0.01
    u = x[None, :] * f + h * th[0] + t * 2.0
    v = x[:, None] * f + h * th[1] + t * -1.0
    # the screen holds float32-rounded values of the linear function: compare within that rounding
    ref = bx * u + by * v
    assert np.max(np.abs(ph - ref)) < 2e-6


def test_dm_single_poke_closed_form_and_subtraction():
    pitch, coup = 0.5, 0.3
    sig = oracle.if_sigma(pitch, coup)
    assert math.exp(-pitch ** 2 / (2 * sig ** 2)) == pytest.approx(coup, rel=1e-14)
    nx = 7
    Cg = np.zeros((nx, nx))
    Cg[2, 4] = 1.3
    n, dx = 30, 0.125
    S = oracle.dm_surface(Cg, pitch, coup, n, dx)
    g = (np.arange(n) - 0.5 * (n - 1)) * dx
    xa, yb = (4 - 3) * pitch, (2 - 3) * pitch
    ref = 1.3 * np.exp(-((g[None, :] - xa) ** 2 + (g[:, None] - yb) ** 2) / (2 * sig ** 2))
    assert np.max(np.abs(S - ref)) < 1e-13
    # subtraction sign: a DM poke lowers the residual phase by the DM surface
    cfg = _small_cfg(alt=0.0, kind="ngs", theta=(0.0, 0.0))
    sim = oracle.Sim(cfg, [np.zeros((256, 256), np.float32)])
    c = np.zeros(sim.n_cmd)
    c[sim.n_cmd // 2] = 2.0
    sim.set_commands(c)
    ph = sim.wfs_phase(0)
    assert ph.min() < -1.0 and ph.max() <= 1e-15


def test_dm_separable_equals_direct_sum_nonsquare():
    rng = np.random.default_rng(4)
    nx, ny, pitch, coup, n, dx = 5, 4, 0.6, 0.25, 14, 0.17
    Cg = rng.standard_normal((ny, nx))
    S = oracle.dm_surface(Cg, pitch, coup, n, dx)
    sig = pitch / math.sqrt(2 * math.log(1 / coup))
    g = (np.arange(n) - 0.5 * (n - 1)) * dx
    ref = np.zeros((n, n))
    for b in range(ny):
        for a in range(nx):
            xa = (a - 0.5 * (nx - 1)) * pitch
            yb = (b - 0.5 * (ny - 1)) * pitch
            for j in range(n):
                for i in range(n):
                    ref[j, i] += Cg[b, a] * math.exp(-((g[i] - xa) ** 2 + (g[j] - yb) ** 2) / (2 * sig * sig))
    assert np.max(np.abs(S - ref)) < 1e-12


# ------------------------------------------------------------------------------------------ science
def test_flat_residual_strehl_one_and_psf_parseval():
    cfg = inputs.scao_tiny()
    sim = oracle.Sim(cfg, [np.zeros((256, 256), np.float32)],
                     np.zeros((inputs.n_commands(cfg), 416), np.float32))
    sim.step(2)
    psf, srl, srk = sim.psf()
    assert srl == pytest.approx(1.0, abs=1e-12) and srk == pytest.approx(1.0, abs=1e-12)
    assert psf.max() == pytest.approx(1.0, abs=1e-12)
    M = psf.shape[0]
    assert np.unravel_index(np.argmax(psf), psf.shape) == (M // 2, M // 2)
    A = oracle.pupil(8.0, 0.0, 128)
    assert psf.sum() == pytest.approx(M * M / A.sum(), rel=1e-10)


def test_sodium_update_equals_configuration():
    """Changing the sodium layer before the first step gives the loop of a configuration created
    with those values (cone projection and elongation both follow)."""
    cfg = inputs.eelt_mcao(n_layers=2, screen_n=1024)
    cfg["wfs"] = cfg["wfs"][:1]
    cfg["science"] = []
    screens = inputs.make_screens(cfg)
    a = oracle.Sim(cfg, screens)
    a.set_sodium(0, 95e3, 14e3)
    b_cfg = dict(cfg, wfs=[dict(cfg["wfs"][0], height=95e3, na_fwhm=14e3)])
    b = oracle.Sim(b_cfg, screens)
    np.testing.assert_array_equal(a.measure(), b.measure())
    with pytest.raises(ValueError):
        a.set_sodium(0, 1.0, 10e3)          # below the layers


def test_marechal_small_phase():
    cfg = inputs.scao_tiny()
    rng = np.random.default_rng(11)
    sig_sci = 0.1
    scr = (rng.standard_normal((256, 256)) * sig_sci * (2.2e-6 / 500e-9)).astype(np.float32)
    sim = oracle.Sim(cfg, [scr], np.zeros((inputs.n_commands(cfg), 416), np.float32))
    ph = sim.wfs_phase(0) * (500e-9 / 2.2e-6)
    A = oracle.pupil(8.0, 0.0, 128)
    p = ph[A > 0]
    var = np.mean((p - p.mean()) ** 2)
    sim.step(1)
    _, srl, _ = sim.psf()
    assert abs(srl - math.exp(-var)) <= var * var
    # the exact definition for the same samples
    assert srl == pytest.approx(abs(np.mean(np.exp(1j * p))) ** 2, rel=1e-12)
    # the Marechal number is exp(-variance) of the same samples
    m_long, m_last = sim.marechal()
    assert m_last == pytest.approx(math.exp(-var), rel=1e-10)
    assert m_long == pytest.approx(math.exp(-var), rel=1e-10)


# ------------------------------------------------------------------------------------------ loop
def _static_aberration_loop():
    """A loop whose only disturbance is a static layer equal to a DM shape c* in the controlled
    space (noise-free, R = -pinv(D)): in the linear regime the reconstructed update is
    dc_k = -(c_k - c*)."""
    cfg = inputs.scao_tiny()
    cfg["layers"][0]["vx"] = 0.0
    zero = [np.zeros((256, 256), np.float32)]
    sim = oracle.Sim(cfg, zero)
    n = sim.n_cmd
    d = 0.05
    D = np.zeros((sim.n_slopes, n))
    for j in range(n):
        c = np.zeros(n)
        c[j] = d
        sim.set_commands(c)
        sp = sim.measure()
        c[j] = -d
        sim.set_commands(c)
        D[:, j] = (sp - sim.measure()) / (2 * d)
    U, S, Vt = np.linalg.svd(D, full_matrices=False)
    keep = S > 1e-2 * S[0]
    R = -(Vt[keep].T / S[keep]) @ U[:, keep].T
    # target commands in the controlled subspace, small enough for the linear regime
    rng = np.random.default_rng(8)
    cstar = Vt[keep].T @ (Vt[keep] @ rng.standard_normal(n)) * 0.01
    sim.set_commands(cstar)
    surf = sim.dm_surface(0)
    scr = np.zeros((256, 256))
    # the DM grid (132 samples) and the layer (256) share the 0.0625 m pitch and both centre
    # on the axis, so the DM shape is written into the layer sample for sample
    off = (256 - 132) // 2
    scr[off:off + 132, off:off + 132] = surf
    loop = oracle.Sim(cfg, [scr.astype(np.float32)], R.astype(np.float32))
    return cfg, loop, cstar


def test_integrator_decay_static_dm_aberration():
    cfg, loop, cstar = _static_aberration_loop()
    g = cfg["gain"]
    for k in range(1, 7):
        loop.step(1)
        err = np.linalg.norm(loop.commands() - cstar) / np.linalg.norm(cstar)
        assert err == pytest.approx((1 - g) ** k, abs=2e-3)


def test_second_order_controller_recursion():
    """Low-pass-filtered integrator (update y_k = (1 - beta) y_{k-1} + beta dc_k, c += g y_k),
    i.e. c_{k+1} = (2 - beta) c_k - (1 - beta) c_{k-1} + g beta dc_k.  With dc_k = -(c_k - c*)
    the error obeys f_{k+1} = (a1 - b0) f_k + a2 f_{k-1}, f_0 = f_{-1} = 1."""
    cfg, loop, cstar = _static_aberration_loop()
    g, beta = 0.5, 0.5
    a1, a2, b0 = 2 - beta, -(1 - beta), g * beta
    loop.set_controller(a1, a2, b0, 0.0)
    f_prev, f = 1.0, 1.0
    for k in range(1, 9):
        loop.step(1)
        f_prev, f = f, (a1 - b0) * f + a2 * f_prev
        err = np.linalg.norm(loop.commands() - cstar) / np.linalg.norm(cstar)
        assert err == pytest.approx(abs(f), abs=3e-3)


def test_controller_integrator_coefficients_match_gain():
    """(a1, a2, b0, b1) = (1, 0, g, 0) is the pure integrator."""
    from _helpers import scao_tiny_inputs
    cfg, screens, R = scao_tiny_inputs()
    a = oracle.Sim(cfg, screens, R)
    b = oracle.Sim(cfg, screens, R)
    b.set_controller(1.0, 0.0, cfg["gain"], 0.0)
    a.step(5)
    b.step(5)
    np.testing.assert_allclose(b.commands(), a.commands(), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------ noise
@pytest.mark.parametrize("x", [-15.9, -10.0, -3.3, -1.0, -0.25, -1e-3, 0.0])
def test_exp_f32_accuracy(x):
    assert oracle.exp_f32(x) == pytest.approx(math.exp(np.float32(x)), rel=4e-7)


def test_log_sincos_f32_accuracy():
    rng = np.random.default_rng(1)
    for u in list(rng.random(300)) + [2 ** -25, 0.125, 0.375, 0.5, 0.625, 0.7071, 0.875, 0.99999994, 1.0]:
        u = float(np.float32(u))
        assert oracle.log_f32(u) == pytest.approx(math.log(u), rel=4e-7, abs=4e-7)
        c, s = oracle.sincos2pi_f32(u)
        assert c == pytest.approx(math.cos(2 * math.pi * u), abs=6e-7)
        assert s == pytest.approx(math.sin(2 * math.pi * u), abs=6e-7)


def test_photon_and_read_noise_independent():
    # each pixel of a pair: photon normal (lambda >= 16, draw B) and read noise (draw A) are
    # independent, so the variances add; the two pixels of a pair are independent of each other
    lam, sig, n = 40.0, 3.0, 100_000
    x = np.array([oracle.noise_pair(lam, lam, sig, i, 5, 2, 11) for i in range(n)], dtype=np.float64)
    var = lam + sig * sig + 2.0 / 12.0   # two roundings to integers
    for a in (0, 1):
        assert x[:, a].mean() == pytest.approx(lam, abs=4 * math.sqrt(var / n))
        assert x[:, a].var() == pytest.approx(var, rel=4 * math.sqrt(2.0 / n) + 0.01)
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 4.0 / math.sqrt(n)
    # a pair with one dim pixel (inversion) and one bright pixel (normal) keeps both laws
    y = np.array([oracle.noise_pair(2.5, 60.0, 0.0, i, 9, 1, 3) for i in range(n)], dtype=np.float64)
    assert y[:, 0].mean() == pytest.approx(2.5, abs=5 * math.sqrt(2.5 / n))
    assert y[:, 0].var() == pytest.approx(2.5, rel=0.03)
    assert y[:, 1].mean() == pytest.approx(60.0, abs=5 * math.sqrt(60.0 / n))
    assert abs(np.corrcoef(y[:, 0], y[:, 1])[0, 1]) < 4.0 / math.sqrt(n)


def test_noise_frame_pairs_within_subaperture_frames():
    # a frame buffer draws pixel pairs (q, q + frame/2) inside each frame: the frame function
    # equals the pair function applied pair by pair
    rng = np.random.default_rng(4)
    lam = rng.uniform(0.0, 40.0, 3 * 64).astype(np.float32)
    fr = oracle.noise_frame(lam, 2.0, 128, 7, 3, 55, frame_px=64)
    for f in range(3):
        for q in range(32):
            a, b = oracle.noise_pair(float(lam[64 * f + q]), float(lam[64 * f + q + 32]), 2.0, 128 + 64 * f + q, 7,
                                     3, 55)
            assert (fr[64 * f + q], fr[64 * f + q + 32]) == (a, b)


@pytest.mark.parametrize("lam", [0.0, 0.7, 5.0, 15.9, 16.0, 40.0, 250.0])
def test_poisson_moments(lam):
    n = 256 * 800
    fr = oracle.noise_frame(np.full(n, lam, np.float32), 0.0, 0, 17, 2, 12345, frame_px=256)
    m, v = fr.mean(), fr.var()
    tol_m = 5 * math.sqrt(max(lam, 1e-3) / n)
    assert abs(m - lam) <= tol_m + 1e-12
    if lam > 0:
        tol_v = 6 * lam * math.sqrt(2.0 / n) + 6 * math.sqrt(lam / n)
        extra = 1.0 / 12.0 if lam >= 16 else 0.0  # rounding of the normal approximation
        assert abs(v - (lam + extra)) <= tol_v + 0.05
    else:
        assert np.all(fr == 0)


def test_read_noise_moments_and_determinism():
    n = 256 * 800
    fr = oracle.noise_frame(np.zeros(n, np.float32), 3.0, 0, 1, 0, 99, frame_px=256)
    assert abs(fr.mean()) < 5 * 3.0 / math.sqrt(n)
    assert fr.var() == pytest.approx(9.0 + 1.0 / 12.0, rel=0.02)
    again = oracle.noise_frame(np.zeros(n, np.float32), 3.0, 0, 1, 0, 99, frame_px=256)
    assert np.array_equal(fr, again)
    other = oracle.noise_frame(np.zeros(n, np.float32), 3.0, 0, 2, 0, 99, frame_px=256)
    assert not np.array_equal(fr, other)
    # the two halves of every frame (the pair partners) are uncorrelated
    f2 = fr.reshape(-1, 2, 128).astype(np.float64)
    assert abs(np.corrcoef(f2[:, 0].ravel(), f2[:, 1].ravel())[0, 1]) < 4.0 / math.sqrt(n / 2)


def test_philox_counter_and_key_dependence():
    base = oracle.philox([0, 0, 0, 0], [0, 0])
    seen = {tuple(base)}
    for i in range(4):
        c = [0, 0, 0, 0]
        c[i] = 1
        o = oracle.philox(c, [0, 0])
        # one flipped input bit changes about half of the 128 output bits
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(o, base))
        assert 40 < flips < 88
        seen.add(tuple(o))
    for i in range(2):
        k = [0, 0]
        k[i] = 1
        seen.add(tuple(oracle.philox([0, 0, 0, 0], k)))
    assert len(seen) == 7
    # uniformity of the top byte over many counters
    words = np.array([oracle.philox([i, 5, 6, 0], [7, 8])[i % 4] for i in range(20000)], dtype=np.uint64)
    hist = np.bincount((words >> 24).astype(np.int64), minlength=256)
    chi2 = (((hist - 20000 / 256) ** 2) / (20000 / 256)).sum()
    assert chi2 < 350


# ------------------------------------------------------------------------------------------ screens
def test_screen_structure_function_matches_von_karman_quadrature():
    from scipy import integrate, special
    n, pixel, r0, L0 = 512, 0.125, 0.2, 25.0
    lags = [2, 4, 8, 16]
    acc = np.zeros(len(lags))
    seeds = range(6)
    for sd in seeds:
        s = inputs.phase_screen(n, pixel, r0, L0, 1000 + sd).astype(np.float64)
        for i, L in enumerate(lags):
            acc[i] += 0.5 * (np.mean((s[:, L:] - s[:, :-L]) ** 2) + np.mean((s[L:, :] - s[:-L, :]) ** 2))
    acc /= len(seeds)
    for i, L in enumerate(lags):
        r = L * pixel

        def f(k):
            return 2 * inputs.von_karman_psd(k, r0, L0) * (1 - special.j0(2 * np.pi * k * r)) * 2 * np.pi * k

        th, _ = integrate.quad(f, 0, np.inf, limit=500)
        assert acc[i] == pytest.approx(th, rel=0.10)
        if r / L0 < 0.02:
            # Kolmogorov limit 6.88 (r/r0)^(5/3) with the leading outer-scale correction
            assert th == pytest.approx(6.88 * (r / r0) ** (5 / 3), rel=0.35)


# ------------------------------------------------------------------ reduced-precision reconstructor
def _torch():
    return pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    torch = _torch()
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1e-3, 4000), rng.normal(0, 30, 4000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0, 1e-40, 3.3e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.bf16_rn(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, ref)
    assert all(oracle.bf16_to_f32(int(h)) == float(torch.tensor([int(h)], dtype=torch.int32).to(torch.int16)
                                                  .view(torch.bfloat16).float()) for h in got[:200])


def test_e4m3_codes_match_torch_and_saturate():
    torch = _torch()
    table = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    for b in range(256):
        v = oracle.e4m3_to_f32(b)
        assert (math.isnan(v) and math.isnan(table[b])) or v == table[b]
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-460, 460, 3000), rng.normal(0, 1e-2, 3000),
                        [2 ** -9, 1.5 * 2 ** -9, 2 ** -10, 2.5 * 2 ** -9, 448.0, 447.0, 440.0, 2 ** -6,
                         0.9375 * 2 ** -6]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_rn_sat(float(v)) for v in x], dtype=np.uint8)
    assert np.array_equal(got, ref)
    # saturation to the largest finite magnitude (torch gives NaN above 464)
    for v in (464.0, 500.0, 1e6, 3e38):
        assert oracle.e4m3_rn_sat(v) == 0x7E and oracle.e4m3_rn_sat(-v) == 0xFE


def test_e4m3_tiny_rows_are_zero_with_unit_scale():
    """A row whose max / 448 is not a normal float gets scale 1 and zero codes (reading: the
    per-row scale must be a normal float; the row's entries are below 448 2^-126).  A row just
    above that threshold keeps its scale and a nonzero largest code."""
    R = np.zeros((3, 16), np.float32)
    R[0, 4] = -4e-40
    R[1, 2] = 3e-36
    R[2, 9] = 6e-36                      # 6e-36 / 448 = 1.3e-38 >= 2^-126
    codes, sc = oracle.quantize_rows(R, oracle.DTYPE_FP8_E4M3)
    assert sc[0] == 1.0 and sc[1] == 1.0
    assert not (codes[0] & 0x7F).any() and not (codes[1] & 0x7F).any()     # +0 or -0 (0x80)
    assert sc[2] == np.float32(np.float32(6e-36) / np.float32(448.0))
    assert codes[2, 9] == 0x7e and np.count_nonzero(codes[2]) == 1
    deq = oracle.dequantize_rows(codes, sc, oracle.DTYPE_FP8_E4M3)
    assert np.all(np.isfinite(deq))


def test_quantize_rows_scales_and_error_bound():
    rng = np.random.default_rng(5)
    R = (rng.normal(0, 1e-2, (37, 301)) * rng.uniform(0.1, 10, (37, 1))).astype(np.float32)
    R[5] = 0.0
    codes, sc = oracle.quantize_rows(R, oracle.DTYPE_FP8_E4M3)
    amax = np.abs(R).max(axis=1)
    assert sc[5] == 1.0 and not codes[5].any()
    nz = amax > 0
    assert np.array_equal(sc[nz], (amax[nz] / np.float32(448.0)).astype(np.float32))
    deq = oracle.dequantize_rows(codes, sc, oracle.DTYPE_FP8_E4M3)
    # half a unit in the last place: 2^-4 relative for normals, 2^-10 scale below 2^-6 scale
    bound = np.maximum(np.abs(R) * 2.0 ** -4, sc[:, None] * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(np.abs(deq - R) <= bound)
    # the largest element of each row maps to +-448 exactly
    i = np.abs(R).argmax(axis=1)
    assert np.all(np.abs(deq[nz, i[nz]]) == pytest.approx(amax[nz], rel=1e-6))
    cb, _ = oracle.quantize_rows(R, oracle.DTYPE_BF16)
    d16 = oracle.dequantize_rows(cb, None, oracle.DTYPE_BF16)
    assert np.all(np.abs(d16 - R) <= np.abs(R) * 2.0 ** -8 * (1 + 1e-6))


@pytest.mark.parametrize("dtype", [1, 2])
def test_reduced_precision_product_is_dequantized_matmul(dtype):
    # one closed-loop step of the 8 m case: the command update equals g * deq(R) @ s
    from tests._helpers import scao_tiny_inputs
    cfg, screens, R = scao_tiny_inputs()
    sim = oracle.Sim(dict(cfg, noise=False), screens, R, r_dtype=dtype)
    sim.step(1)
    s = sim.slopes()
    codes, sc = oracle.quantize_rows(R, dtype)
    deq = oracle.dequantize_rows(codes, sc, dtype)
    np.testing.assert_allclose(sim.commands(), cfg["gain"] * (deq @ s), rtol=1e-12, atol=1e-15)
    sim.close()


# ---- phase screens by the FFT method ("The atmospheric layers generation") ----------------

def _d_von_karman(r, r0, L0):
    """Von Karman phase structure function for PSD 0.023 r0^-5/3 (f^2 + f0^2)^-11/6 (f in
    cycles/m): D(r) = 4 pi 0.023 r0^-5/3 int_0^inf f (1 - J0(2 pi f r)) (f^2 + f0^2)^-11/6 df,
    the Bessel part by the Hankel transform int_0^inf x J0(bx) (x^2 + a^2)^-(mu+1) dx
    = (b / a)^mu K_mu(ab) / (2^mu Gamma(mu + 1)), mu = 5/6."""
    from scipy.special import gamma, kv
    f0 = 1.0 / L0
    b = 2.0 * np.pi * r
    return 4.0 * np.pi * 0.023 * r0 ** (-5.0 / 3.0) * (
        0.6 * f0 ** (-5.0 / 3.0) - f0 ** (-5.0 / 6.0) * b ** (5.0 / 6.0) * kv(5.0 / 6.0, b * f0)
        / (2.0 ** (5.0 / 6.0) * gamma(11.0 / 6.0)))


def test_von_karman_closed_form_reaches_kolmogorov():
    # L0 -> infinity and r << L0: D -> 6.88 (r / r0)^(5/3); the outer-scale correction falls
    # off as (r / L0)^(1/3) and the 0.023 constant is 6.88's rounded counterpart (0.5 % apart)
    r0 = 0.15
    for r in (0.05, 0.1, 0.3):
        assert _d_von_karman(r, r0, 1e7) == pytest.approx(6.88 * (r / r0) ** (5.0 / 3.0), rel=0.01)


@pytest.mark.parametrize("n,pixel", [(1024, 0.05), (2048, 0.05)])
def test_screen_spectrum_matches_von_karman_structure_function(n, pixel):
    # the generator's amplitudes give the expected structure function sum a_k^2 2(1 - cos);
    # on a screen much larger than L0 it is the von Karman D(r) up to the frequencies above
    # Nyquist (a few % at 2 samples, < 0.5 % from 10 samples on)
    r0, L0 = 0.15, 10.0
    for r_px, tol in ((2, 0.04), (10, 0.005), (40, 0.002)):
        d = oracle.screen_structure_function(n, pixel, r0, L0, r_px)
        assert d == pytest.approx(_d_von_karman(r_px * pixel, r0, L0), rel=tol)
    a = oracle.screen_amp(n, pixel, r0, L0)
    assert a[0, 0] == 0.0
    # Hermitian-symmetric amplitudes: a(-k) = a(k)
    assert np.array_equal(a[1:, 1:], a[1:, 1:][::-1, ::-1]) or n % 2 == 0


def test_screen_coefficients_are_standard_complex_normal():
    n, pixel, r0, L0 = 128, 0.1, 0.15, 3.2
    a = oracle.screen_amp(n, pixel, r0, L0)
    m = a > 0
    z = np.concatenate([oracle.screen_coeffs(n, pixel, r0, L0, s)[m] / a[m] for s in range(20)])
    assert abs(z.real.mean()) < 0.01 and abs(z.imag.mean()) < 0.01
    assert z.real.var() == pytest.approx(1.0, abs=0.012) and z.imag.var() == pytest.approx(1.0, abs=0.012)
    assert abs(np.mean(z.real * z.imag)) < 0.01
    assert np.mean(z.real ** 4) / np.mean(z.real ** 2) ** 2 == pytest.approx(3.0, abs=0.05)
    # draws differ across seeds and grid positions
    c0 = oracle.screen_coeffs(n, pixel, r0, L0, 0)
    c1 = oracle.screen_coeffs(n, pixel, r0, L0, 1)
    assert abs(np.corrcoef(c0[m].real / a[m], c1[m].real / a[m])[0, 1]) < 0.05


def test_screen_statistics_match_expected_moments():
    # exact invariants and ensemble moments of Re sum_k c_k e^{2 pi i k.x/n}: zero mean over
    # the grid (no DC term), variance sum a_k^2, structure function sum a_k^2 2 (1 - cos)
    n, pixel, r0, L0 = 128, 0.1, 0.15, 3.2
    S = np.array([oracle.phase_screen(n, pixel, r0, L0, s) for s in range(40)])
    rms = S.std()
    assert np.abs(S.mean(axis=(1, 2))).max() < 1e-12 * rms
    var = np.sum(oracle.screen_amp(n, pixel, r0, L0) ** 2)
    assert S.var(axis=(1, 2)).mean() == pytest.approx(var, rel=0.1)
    for r_px, tol in ((1, 0.03), (4, 0.05)):
        want = oracle.screen_structure_function(n, pixel, r0, L0, r_px)
        for ax in (1, 2):
            got = np.mean((np.roll(S, -r_px, axis=ax) - S) ** 2)
            assert got == pytest.approx(want, rel=tol)
    # isotropy: the x and y lags come from the same amplitudes
    a = oracle.screen_amp(n, pixel, r0, L0)
    assert np.allclose(a, a.T)


# ---- derivatives of the noise-free sensing (interaction matrix by the Jacobian) -------------

@pytest.mark.parametrize("sigma", [0.0, 2.0])
def test_subap_jacobian_fd_invariants(sigma):
    # the centroid ignores piston (the derivative sums to zero over the subaperture), samples of
    # zero amplitude do not act, and halving the step changes the central difference by O(h^2)
    rng = np.random.default_rng(3)
    amp = np.ones((8, 8))
    amp[0, 0] = 0.0
    amp[0, 7] = 0.5
    ph = rng.normal(0.0, 0.5, (8, 8))
    J1 = oracle.subap_jacobian_fd(amp, ph, 16, 2, sigma, (0.6, 0.8), h=1e-4)
    J2 = oracle.subap_jacobian_fd(amp, ph, 16, 2, sigma, (0.6, 0.8), h=5e-5)
    scale = np.abs(J1).max()
    assert scale > 0.01
    assert np.abs(J1 - J2).max() <= 1e-7 * scale
    for a in (0, 1):
        assert abs(J1[a].sum()) <= 1e-8 * scale
    assert np.all(J1[:, 0, 0] == 0.0)
    # a phase ramp along x moves the x centroid, not (to first order, for a mirror-symmetric
    # pupil and flat wavefront) the y one
    flat = oracle.subap_jacobian_fd(np.ones((8, 8)), np.zeros((8, 8)), 16, 2, 0.0, (1.0, 0.0), h=1e-4)
    ramp = np.tile(np.arange(8) - 3.5, (8, 1))
    assert np.sum(flat[0] * ramp) > 0.1
    assert abs(np.sum(flat[1] * ramp)) <= 1e-8 * abs(np.sum(flat[0] * ramp))


def test_interaction_matrix_fd_is_the_derivative():
    # central differences at h and h/2 agree to O(h^2); the first-order prediction
    # s(c + e d) - s(c) - e D d shrinks like e^2 (relative error like e), which a wrong D breaks
    from tests._helpers import mcao_small
    cfg = mcao_small()
    o = oracle.Sim(cfg, inputs.make_screens(cfg))
    rng = np.random.default_rng(1)
    o.set_commands(rng.normal(0.0, 0.3, o.n_cmd))
    D1 = oracle.jacobian_fd(o, 1e-3)
    D2 = oracle.jacobian_fd(o, 5e-4)
    n = np.linalg.norm
    assert n(D1 - D2) <= 1e-7 * n(D1)
    c0 = o.commands()
    s0 = o.measure()
    d = rng.normal(0.0, 1.0, o.n_cmd)
    rel = []
    for eps in (1e-2, 2.5e-3):
        o.set_commands(c0 + eps * d)
        rel.append(n(o.measure() - s0 - eps * (D1 @ d)) / n(eps * (D1 @ d)))
    assert rel[0] < 2e-3
    assert 2.5 < rel[0] / rel[1] < 6.0      # linear in eps: ratio 4
    o.close()


# ---- misregistered DM: the surface of the DM moved as a rigid body ---------------------------

def test_misregistered_surface_identities():
    # identity transform = the factorised surface; a quarter turn = the aligned surface of the
    # rotated command grid; a shift by whole surface samples = the shifted surface; a
    # magnification of 2 on an odd grid = the aligned surface at half the coordinates
    rng = np.random.default_rng(0)
    n, pitch, cp, sn, dx = 9, 0.5, 0.3, 41, 0.125
    C_ = rng.normal(size=(n, n))
    S0 = oracle.dm_surface(C_, pitch, cp, sn, dx)
    tol = 1e-12 * np.abs(S0).max()
    assert np.abs(oracle.dm_surface_misreg(C_, pitch, cp, sn, dx) - S0).max() <= tol
    Cr = np.zeros_like(C_)
    for b in range(n):
        for a in range(n):
            Cr[a, n - 1 - b] = C_[b, a]          # actuator (x_a, y_b) moves to (-y_b, x_a)
    S90 = oracle.dm_surface_misreg(C_, pitch, cp, sn, dx, rotation=np.pi / 2)
    assert np.abs(S90 - oracle.dm_surface(Cr, pitch, cp, sn, dx)).max() <= tol
    Ssh = oracle.dm_surface_misreg(C_, pitch, cp, sn, dx, shift=(3 * dx, -2 * dx))
    assert np.abs(Ssh[:-2, 3:] - S0[2:, :-3]).max() <= tol
    Sm = oracle.dm_surface_misreg(C_, pitch, cp, sn, dx, magnification=2.0)
    i = np.arange(0, sn, 2)
    h = 20 + (i - 20) // 2
    assert np.abs(Sm[np.ix_(i, i)] - S0[np.ix_(h, h)]).max() <= tol


def test_misregistration_moves_the_measurement():
    # identity misregistration leaves the slopes unchanged bit for bit; a shift changes them;
    # shifting back restores them
    from tests._helpers import mcao_small
    cfg = mcao_small()
    o = oracle.Sim(cfg, inputs.make_screens(cfg))
    o.set_commands(np.random.default_rng(2).normal(0.0, 0.3, o.n_cmd))
    s0 = o.measure()
    o.set_misregistration(0, 0.0, 0.0, 0.0, 1.0)
    assert np.array_equal(o.measure(), s0)
    o.set_misregistration(0, 0.3, -0.2, 0.01, 1.01)
    assert np.abs(o.measure() - s0).max() > 1e-3
    o.set_misregistration(0, 0.0, 0.0, 0.0, 1.0)
    assert np.array_equal(o.measure(), s0)
    with pytest.raises(ValueError):
        o.set_misregistration(0, 0.0, 0.0, 0.0, 0.0)
    o.close()


# ------------------------------------------------------------------------------------------ control matrix
def test_tikhonov_equals_svd_filter_form():
    """The regularised normal equations equal the SVD filter form -V diag(s / (s^2 + lam)) U^T, an
    independent route (a dropped lambda, a transposed D or a lost sign fails here), and lam is
    alpha times the mean diagonal of D^T D."""
    rng = np.random.default_rng(31)
    D = rng.standard_normal((90, 40)) @ np.diag(np.logspace(0, -4, 40))
    R, lam = oracle.tikhonov_reconstructor(D, 1e-3)
    assert lam == pytest.approx(1e-3 * np.sum(D * D) / 40, rel=1e-13)
    U, sv, Vt = np.linalg.svd(D, full_matrices=False)
    ref = -(Vt.T * (sv / (sv * sv + lam))) @ U.T
    assert np.max(np.abs(R - ref)) <= 1e-10 * np.max(np.abs(ref))
    res = (D.T @ D + lam * np.eye(40)) @ R + D.T
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(D))


def test_tikhonov_limits():
    """alpha -> 0 with full column rank gives -pinv(D); orthogonal columns of norm c give the
    closed form -c / (c^2 + lam) per column direction."""
    rng = np.random.default_rng(32)
    D = rng.standard_normal((60, 25))
    R0, _ = oracle.tikhonov_reconstructor(D, 0.0)
    assert np.max(np.abs(R0 + np.linalg.pinv(D))) <= 1e-10
    Q, _ = np.linalg.qr(rng.standard_normal((60, 25)))
    c = 3.0
    R1, lam = oracle.tikhonov_reconstructor(c * Q, 0.1)
    assert lam == pytest.approx(0.1 * c * c, rel=1e-13)
    assert np.max(np.abs(R1 + (c / (c * c + lam)) * Q.T)) <= 1e-12


def test_workload_sizes():
    # the two configurations' sizes: 208 valid subapertures (416 slopes) and a 17 x 17 DM on the
    # 8 m case; 4632 valid subapertures per laser star, 55 608 slopes and 8051 commands on the
    # 39 m case (zero screens: only the geometry is exercised)
    cfg = inputs.scao_tiny()
    o = oracle.Sim(cfg, [np.zeros((l["n"], l["n"]), np.float32) for l in cfg["layers"]])
    assert (o.n_valid(0), o.n_slopes) == (208, 416)
    assert cfg["dms"][0]["nx"] == 17 and o.n_cmd == inputs.n_commands(cfg)
    o.close()
    big = inputs.eelt_mcao(screen_n=64)
    o = oracle.Sim(big, [np.zeros((l["n"], l["n"]), np.float32) for l in big["layers"]])
    assert [o.n_valid(w) for w in range(6)] == [4632] * 6
    assert o.n_slopes == 55608 and o.n_cmd == 8051 == inputs.n_commands(big)
    o.close()
