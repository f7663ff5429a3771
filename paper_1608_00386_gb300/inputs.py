"""Seeded synthetic inputs: system configurations, phase screens and reconstructors.

This module only describes and draws inputs; it holds none of the wavefront-sensing or control
arithmetic.  Both the CUDA library (through the binding) and the CPU oracle (through the tests)
read the same dictionaries and arrays produced here.

Two configurations are defined:

* ``scao_tiny``: 8 m unobstructed pupil, one on-axis natural guide star, one von Karman layer
  (r0 = 0.15 m at 500 nm, L0 = 25 m, 10 m/s) on a 256 x 256 screen at 0.0625 m, 16 x 16
  Shack-Hartmann subapertures of 8 x 8 samples, 16 x 16 FFT, 8 x 8 detector pixels, one 17 x 17
  Gaussian-influence DM (coupling 0.3), integrator gain 0.5, dt = 2 ms.
* ``eelt_mcao``: 39 m pupil with 28 % obstruction, 10 layers (synthetic profile 0-20 km,
  r0 = 0.157 m, winds 5-30 m/s) on 2048 x 2048 screens at 0.0609375 m, six sodium laser guide
  stars on a 45 arcsec ring at 90 km (80 x 80 subapertures of 8 x 8 samples, 32 x 32 FFT,
  16 x 16 detector pixels, 10 km FWHM sodium layer, launch at the pupil centre), three natural
  guide stars at 60 arcsec with 2 x 2 low-order sensors (32 samples per subaperture, 64 x 64
  FFT, 4 x 4 binning), three DMs at 0 / 4 / 12.7 km with about 5300 / 1500 / 1300 actuators.

The paper ("The numerical simulation tool for the MAORY multiconjugate adaptive optics system",
arXiv:1608.00386) gives the architecture (six LGS Shack-Hartmann sensors, three NGS low-order
sensors, three DMs; MAORY subsection of the introduction) but no turbulence profile; the
ten-layer profile here is synthetic.
"""
from __future__ import annotations

import math

import numpy as np

ARCSEC = math.pi / 180.0 / 3600.0

# ------------------------------------------------------------------------------------------
# phase screens
# ------------------------------------------------------------------------------------------


def von_karman_psd(kappa: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Phase power spectrum 0.023 r0^-5/3 (k^2 + 1/L0^2)^-11/6, k in cycles per metre."""
    return 0.023 * r0 ** (-5.0 / 3.0) * (kappa * kappa + 1.0 / (L0 * L0)) ** (-11.0 / 6.0)


def phase_screen(n: int, pixel: float, r0: float, L0: float, seed: int) -> np.ndarray:
    """Periodic n x n von Karman screen (rad at the wavelength r0 refers to) by the FFT method.

    Complex Gaussian coefficients weighted by sqrt(PSD) dk on the discrete frequency grid,
    zero mean (DC removed), real part kept.  Returns float32, row-major [y][x].
    """
    rng = np.random.default_rng(seed)
    dk = 1.0 / (n * pixel)
    f = np.fft.fftfreq(n, d=pixel)
    kx, ky = np.meshgrid(f, f)
    amp = np.sqrt(von_karman_psd(np.hypot(kx, ky), r0, L0)) * dk
    amp[0, 0] = 0.0
    c = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * amp
    scr = np.real(np.fft.ifft2(c)) * (n * n)
    return scr.astype(np.float32)


def make_screens(cfg: dict, realization: int = 0) -> list[np.ndarray]:
    """Screens of every layer of a configuration (each layer carries its own r0 and seed);
    realization r draws independent screens (layer seed + 1000 r)."""
    out = []
    for lay in cfg["layers"]:
        r0_l = lay["r0"]
        out.append(phase_screen(lay["n"], lay["pixel"], r0_l, lay["L0"], lay["seed"] + 1000 * realization))
    return out


def shifted_screens(screens: list[np.ndarray], realization: int, n_real: int) -> list[np.ndarray]:
    """Screens of realization r as the given screens rolled by r n / n_real samples along x
    (periodic screens: same statistics, distinct samples; no FFT per realization)."""
    out = []
    for s in screens:
        n = s.shape[1]
        out.append(np.roll(s, (realization * n) // max(n_real, 1), axis=1))
    return out


# ------------------------------------------------------------------------------------------
# DM geometry
# ------------------------------------------------------------------------------------------


def _metapupil_radius(cfg: dict, alt: float) -> float:
    """Largest radius, at altitude alt, of the beam footprint of any guide star or science
    direction: (D/2)(1 - alt/H) + alt |theta|, H infinite for stars at infinity."""
    r = 0.0
    for w in cfg["wfs"]:
        f = 1.0 - alt / w["height"] if w["type"] == "lgs" else 1.0
        r = max(r, 0.5 * cfg["D"] * f + alt * math.hypot(*w["theta"]))
    for s in cfg["science"]:
        r = max(r, 0.5 * cfg["D"] + alt * math.hypot(*s["theta"]))
    return r


def dm_spec(cfg: dict, alt: float, pitch: float, coupling: float = 0.3, nx: int | None = None) -> dict:
    """Fried-geometry actuator grid at pitch, valid within the metapupil radius plus one pitch;
    the surface grid samples the metapupil at the finest guide-star pupil pitch with a margin
    of two samples (even size, so an on-axis ground DM aligns with the pupil samples)."""
    rm = _metapupil_radius(cfg, alt)
    if nx is None:
        nx = 2 * int(math.ceil((rm + pitch) / pitch)) + 1
    a = (np.arange(nx) - 0.5 * (nx - 1)) * pitch
    X, Y = np.meshgrid(a, a)
    valid = ((X * X + Y * Y) <= (rm + pitch) ** 2).astype(np.uint8)
    dx = min(cfg["D"] / (w["n_sub"] * w["n_px"]) for w in cfg["wfs"])
    surf_n = 2 * int(math.ceil(rm / dx)) + 4
    return {"alt": alt, "pitch": pitch, "coupling": coupling, "nx": nx, "ny": nx,
            "valid": valid, "surf_n": surf_n, "surf_dx": dx}


# ------------------------------------------------------------------------------------------
# configurations
# ------------------------------------------------------------------------------------------


def _wfs(kind, theta, n_sub, n_px, n_fft, n_bin, lam, n_photons, height=0.0, na_fwhm=0.0,
         read_noise=3.0, valid_thr=0.5, launch=(0.0, 0.0)):
    return {"type": kind, "theta": tuple(theta), "height": height, "n_sub": n_sub, "n_px": n_px,
            "n_fft": n_fft, "n_bin": n_bin, "lambda": lam, "n_photons": n_photons,
            "read_noise": read_noise, "valid_thr": valid_thr, "na_fwhm": na_fwhm,
            "launch": tuple(launch)}


def scao_tiny(noise: bool = False, seed: int = 7) -> dict:
    """8 m single-conjugate case: 1 NGS, 1 layer, 16 x 16 subapertures, 17 x 17 DM."""
    cfg = {
        "name": "scao_tiny_8m",
        "D": 8.0, "obstruction": 0.0, "lambda_ref": 500e-9,
        "dt": 2e-3, "gain": 0.5, "seed": seed, "noise": bool(noise), "psf_every": 1,
        "n_steps": 100,
        "wfs": [_wfs("ngs", (0.0, 0.0), 16, 8, 16, 2, 500e-9, 500.0)],
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 128, "pad": 2}],
        "layers": [{"n": 256, "pixel": 0.0625, "alt": 0.0, "vx": 10.0, "vy": 0.0,
                    "r0": 0.15, "L0": 25.0, "seed": 1}],
    }
    cfg["dms"] = [dm_spec(cfg, 0.0, 0.5, 0.3, nx=17)]
    return cfg


EELT_HEIGHTS_KM = [0.0, 0.6, 1.2, 2.5, 4.0, 6.0, 8.5, 11.0, 14.0, 20.0]
EELT_FRACTIONS = [0.5, 0.08, 0.07, 0.07, 0.06, 0.06, 0.05, 0.04, 0.04, 0.03]


def eelt_mcao(noise: bool = False, seed: int = 7, screen_n: int = 2048, n_layers: int = 10) -> dict:
    """39 m MCAO case: 6 LGS (80 x 80) + 3 NGS (2 x 2), 10 layers, 3 DMs."""
    D = 39.0
    dx = D / 640.0
    fr = np.array(EELT_FRACTIONS[:n_layers], dtype=np.float64)
    fr = fr / fr.sum()
    winds = np.linspace(5.0, 30.0, 10)[:n_layers]
    r0 = 0.157
    layers = []
    for l in range(n_layers):
        ang = math.radians(36.0 * l)
        layers.append({"n": screen_n, "pixel": dx, "alt": EELT_HEIGHTS_KM[l] * 1e3,
                       "vx": float(winds[l] * math.cos(ang)), "vy": float(winds[l] * math.sin(ang)),
                       "r0": float(r0 * fr[l] ** (-3.0 / 5.0)), "L0": 25.0, "seed": 1 + l})
    wfs = []
    for i in range(6):
        a = math.radians(60.0 * i)
        wfs.append(_wfs("lgs", (45 * ARCSEC * math.cos(a), 45 * ARCSEC * math.sin(a)), 80, 8, 32, 2,
                        589e-9, 1000.0, height=90e3, na_fwhm=10e3))
    for a_deg in (30.0, 150.0, 270.0):
        a = math.radians(a_deg)
        wfs.append(_wfs("ngs", (60 * ARCSEC * math.cos(a), 60 * ARCSEC * math.sin(a)), 2, 32, 64, 4,
                        1.65e-6, 500.0))
    cfg = {
        "name": "eelt_mcao_6lgs",
        "D": D, "obstruction": 0.28, "lambda_ref": 500e-9,
        "dt": 2e-3, "gain": 0.5, "seed": seed, "noise": bool(noise), "psf_every": 1,
        "n_steps": 1000,
        "wfs": wfs,
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 640, "pad": 2}],
        "layers": layers,
    }
    cfg["dms"] = [dm_spec(cfg, 0.0, 0.4875, 0.3, nx=81),
                  dm_spec(cfg, 4000.0, 1.0, 0.3),
                  dm_spec(cfg, 12700.0, 1.19, 0.3)]
    return cfg


def mcao_20m(noise: bool = False, seed: int = 7) -> dict:
    """20 m MCAO case: 3 LGS (40 x 40, 8 px, FFT 32, bin 2, elongated) + 1 NGS 2 x 2, 5 layers
    of 1024^2, 2 DMs (0 and 8 km)."""
    D = 20.0
    dx = D / 320.0
    heights = [0.0, 1.0e3, 3.0e3, 6.0e3, 12.0e3]
    frac = np.array([0.5, 0.15, 0.15, 0.1, 0.1])
    layers = []
    for l, h in enumerate(heights):
        ang = math.radians(50.0 * l)
        v = 6.0 + 4.0 * l
        layers.append({"n": 1024, "pixel": dx, "alt": h, "vx": float(v * math.cos(ang)), "vy": float(v * math.sin(ang)),
                       "r0": float(0.157 * frac[l] ** (-3.0 / 5.0)), "L0": 25.0, "seed": 21 + l})
    wfs = []
    for i in range(3):
        a = math.radians(120.0 * i)
        wfs.append(_wfs("lgs", (30 * ARCSEC * math.cos(a), 30 * ARCSEC * math.sin(a)), 40, 8, 32, 2, 589e-9, 1000.0,
                        height=90e3, na_fwhm=10e3))
    wfs.append(_wfs("ngs", (40 * ARCSEC, 0.0), 2, 32, 64, 4, 1.65e-6, 500.0))
    cfg = {
        "name": "mcao_20m_3lgs",
        "D": D, "obstruction": 0.2, "lambda_ref": 500e-9,
        "dt": 2e-3, "gain": 0.5, "seed": seed, "noise": bool(noise), "psf_every": 1, "n_steps": 1000,
        "wfs": wfs,
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 320, "pad": 2}],
        "layers": layers,
    }
    cfg["dms"] = [dm_spec(cfg, 0.0, 0.5, 0.3), dm_spec(cfg, 8000.0, 1.0, 0.3)]
    return cfg


def mixed_configs(n: int, noise: bool = True) -> list[dict]:
    """n configurations of mixed sizes for group stepping: cycles through the 8 m single-NGS case
    (16 x 16 subapertures, 1 layer) and the 20 m 3-LGS case (40 x 40, 5 layers), each with its
    own noise seed."""
    out = []
    for i in range(n):
        cfg = scao_tiny(noise=noise, seed=100 + i) if i % 2 == 0 else mcao_20m(noise=noise, seed=100 + i)
        out.append(cfg)
    return out


def n_commands(cfg: dict) -> int:
    return int(sum(int(d["valid"].sum()) for d in cfg["dms"]))


def random_reconstructor(n_cmd: int, n_slopes: int, sigma: float, seed: int) -> np.ndarray:
    """Dense float32 [n_cmd][n_slopes] matrix with N(0, sigma^2) entries (throughput runs)."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_cmd, n_slopes), dtype=np.float32)
    for i0 in range(0, n_cmd, 512):
        i1 = min(n_cmd, i0 + 512)
        out[i0:i1] = rng.standard_normal((i1 - i0, n_slopes), dtype=np.float32) * np.float32(sigma)
    return out
