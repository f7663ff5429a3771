"""FP64 CPU oracle of the MCAO wavefront-sensing-and-control step (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import this
package.  It wraps ``mcao_oracle.c`` (plain C, double precision, OpenMP over independent
subapertures and matrix rows) through ctypes and shares no code with the CUDA library.

The C file's header lists what each function computes and which passage of arXiv:1608.00386
(or which stated reading) it follows.  ``build()`` compiles it with ``-ffp-contract=off`` so
that the float noise sampler keeps its written operation order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcao_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)
_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)


class _Wfs(C.Structure):
    _fields_ = [("type", C.c_int), ("n_sub", C.c_int), ("n_px", C.c_int), ("n_fft", C.c_int),
                ("n_bin", C.c_int), ("pad_", C.c_int),
                ("theta_x", C.c_double), ("theta_y", C.c_double), ("height", C.c_double),
                ("lambda_", C.c_double), ("n_photons", C.c_double), ("read_noise", C.c_double),
                ("valid_thr", C.c_double), ("na_fwhm", C.c_double),
                ("launch_x", C.c_double), ("launch_y", C.c_double)]


class _Sci(C.Structure):
    _fields_ = [("n_px", C.c_int), ("pad", C.c_int),
                ("theta_x", C.c_double), ("theta_y", C.c_double), ("lambda_", C.c_double)]


class _Layer(C.Structure):
    _fields_ = [("n", C.c_int), ("pad_", C.c_int), ("pixel", C.c_double), ("alt", C.c_double),
                ("vx", C.c_double), ("vy", C.c_double), ("phase", _fp)]


class _Dm(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("surf_n", C.c_int), ("pad_", C.c_int),
                ("alt", C.c_double), ("pitch", C.c_double), ("coupling", C.c_double),
                ("surf_dx", C.c_double), ("valid", C.POINTER(C.c_uint8))]


class _Config(C.Structure):
    _fields_ = [("D", C.c_double), ("obstruction", C.c_double), ("lambda_ref", C.c_double),
                ("dt", C.c_double), ("gain", C.c_double), ("seed", C.c_uint64),
                ("noise", C.c_int), ("psf_every", C.c_int),
                ("n_wfs", C.c_int), ("n_sci", C.c_int), ("n_layers", C.c_int), ("n_dms", C.c_int),
                ("wfs", C.POINTER(_Wfs)), ("sci", C.POINTER(_Sci)), ("layers", C.POINTER(_Layer)),
                ("dms", C.POINTER(_Dm)), ("n_cmd", C.c_int), ("n_slopes", C.c_int),
                ("R", _fp), ("s_ref", _fp), ("r_dtype", C.c_int)]

DTYPE_F32, DTYPE_BF16, DTYPE_FP8_E4M3 = 0, 1, 2


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_fft1.argtypes = [C.c_int, _dp, _dp, C.c_int]
        L.orc_fft2.argtypes = [C.c_int, _dp, _dp, C.c_int]
        L.orc_pupil.argtypes = [C.c_double, C.c_double, C.c_int, _dp]
        L.orc_valid_subaps.argtypes = [_dp, C.c_int, C.c_int, C.c_double, _ip, _dp]
        L.orc_valid_subaps.restype = C.c_int
        L.orc_bilinear_periodic.argtypes = [_dp, C.c_int, C.c_double, C.c_double]
        L.orc_bilinear_periodic.restype = C.c_double
        L.orc_bilinear_clamped.argtypes = [_dp, C.c_int, C.c_double, C.c_double]
        L.orc_bilinear_clamped.restype = C.c_double
        L.orc_if_sigma.argtypes = [C.c_double, C.c_double]
        L.orc_if_sigma.restype = C.c_double
        L.orc_dm_surface.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, _dp, _dp]
        L.orc_sh_image.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_bin.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.orc_cog.argtypes = [C.c_int, _dp, _dp, _dp]
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_uniform_f32.argtypes = [C.c_uint32]
        L.orc_uniform_f32.restype = C.c_float
        L.orc_sincos2pi_f32.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.orc_sincos2pi_f32.restype = None
        for nm in ("orc_exp_f32", "orc_log_f32"):
            getattr(L, nm).argtypes = [C.c_float]
            getattr(L, nm).restype = C.c_float
        L.orc_bf16_rn.argtypes = [C.c_float]
        L.orc_bf16_rn.restype = C.c_uint16
        L.orc_bf16_to_f32.argtypes = [C.c_uint16]
        L.orc_bf16_to_f32.restype = C.c_float
        L.orc_e4m3_rn_sat.argtypes = [C.c_float]
        L.orc_e4m3_rn_sat.restype = C.c_uint8
        L.orc_e4m3_to_f32.argtypes = [C.c_uint8]
        L.orc_e4m3_to_f32.restype = C.c_float
        L.orc_quantize_rows.argtypes = [_fp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, _fp]
        L.orc_set_controller.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_marechal.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.orc_set_sodium.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        L.orc_set_misregistration.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_dm_surface_misreg.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                            C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
        L.orc_get_elongation.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.orc_screen_amp.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_screen_coeffs.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64, _dp, _dp]
        L.orc_set_sodium.restype = C.c_int
        L.orc_noise_pair.argtypes = [C.c_float, C.c_float, C.c_float, C.c_uint32, C.c_uint32, C.c_uint32,
                                     C.c_uint64, _i32p, _i32p]
        L.orc_noise_frame.argtypes = [_fp, C.c_int, C.c_int, C.c_float, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint64, _i32p]
        L.orc_create.argtypes = [C.POINTER(_Config)]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_measure.argtypes = [C.c_void_p, _dp]
        for nm in ("orc_n_cmd", "orc_n_slopes"):
            getattr(L, nm).argtypes = [C.c_void_p]
            getattr(L, nm).restype = C.c_int
        L.orc_n_valid.argtypes = [C.c_void_p, C.c_int]
        L.orc_n_valid.restype = C.c_int
        L.orc_step_index.argtypes = [C.c_void_p]
        L.orc_step_index.restype = C.c_long
        L.orc_set_step_index.argtypes = [C.c_void_p, C.c_long]
        L.orc_get_valid.argtypes = [C.c_void_p, C.c_int, _ip]
        L.orc_get_slopes.argtypes = [C.c_void_p, _dp]
        L.orc_get_commands.argtypes = [C.c_void_p, _dp]
        L.orc_set_commands.argtypes = [C.c_void_p, _dp]
        L.orc_get_dm_surface.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_wfs_phase.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_get_frames.argtypes = [C.c_void_p, C.c_int, _fp, _i32p]
        L.orc_get_psf.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp]
        L.orc_num_threads.restype = C.c_int
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ------------------------------------------------------------------------------------------
# stage functions
# ------------------------------------------------------------------------------------------

def fft1(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    re = np.ascontiguousarray(np.real(x), dtype=np.float64).copy()
    im = np.ascontiguousarray(np.imag(x), dtype=np.float64).copy()
    lib().orc_fft1(len(re), _ptr(re, C.c_double), _ptr(im, C.c_double), int(inverse))
    return re + 1j * im


def fft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    re = np.ascontiguousarray(np.real(x), dtype=np.float64).copy()
    im = np.ascontiguousarray(np.imag(x), dtype=np.float64).copy()
    lib().orc_fft2(re.shape[0], _ptr(re, C.c_double), _ptr(im, C.c_double), int(inverse))
    return re + 1j * im


def pupil(D: float, obstruction: float, n: int) -> np.ndarray:
    A = np.zeros((n, n))
    lib().orc_pupil(D, obstruction, n, _ptr(A, C.c_double))
    return A


def valid_subaps(A: np.ndarray, n_sub: int, n_px: int, thr: float):
    A = np.ascontiguousarray(A, dtype=np.float64)
    v = np.zeros(n_sub * n_sub, dtype=np.int32)
    f = np.zeros(n_sub * n_sub)
    cnt = lib().orc_valid_subaps(_ptr(A, C.c_double), n_sub, n_px, thr, _ptr(v, C.c_int), _ptr(f, C.c_double))
    return cnt, v.reshape(n_sub, n_sub), f.reshape(n_sub, n_sub)


def bilinear_periodic(s: np.ndarray, fx: float, fy: float) -> float:
    s = np.ascontiguousarray(s, dtype=np.float64)
    return lib().orc_bilinear_periodic(_ptr(s, C.c_double), s.shape[0], fx, fy)


def bilinear_clamped(s: np.ndarray, fx: float, fy: float) -> float:
    """Bilinear sample of a bounded n x n grid (index clamped into [0, n-1]), the rule used for
    DM surfaces; s is [y][x]."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    return lib().orc_bilinear_clamped(_ptr(s, C.c_double), s.shape[0], fx, fy)


def if_sigma(pitch: float, coupling: float) -> float:
    return lib().orc_if_sigma(pitch, coupling)


def dm_surface(cmd_grid: np.ndarray, pitch: float, coupling: float, surf_n: int, surf_dx: float) -> np.ndarray:
    Cg = np.ascontiguousarray(cmd_grid, dtype=np.float64)
    S = np.zeros((surf_n, surf_n))
    lib().orc_dm_surface(Cg.shape[1], Cg.shape[0], pitch, coupling, surf_n, surf_dx,
                         _ptr(Cg, C.c_double), _ptr(S, C.c_double))
    return S


def sh_image(amp: np.ndarray, phase: np.ndarray, n_fft: int, sigma_pix: float = 0.0,
             direction=(1.0, 0.0)) -> np.ndarray:
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    phase = np.ascontiguousarray(phase, dtype=np.float64)
    img = np.zeros((n_fft, n_fft))
    lib().orc_sh_image(amp.shape[0], n_fft, _ptr(amp, C.c_double), _ptr(phase, C.c_double),
                       sigma_pix, direction[0], direction[1], _ptr(img, C.c_double))
    return img


def dm_surface_misreg(cmd_grid: np.ndarray, pitch: float, coupling: float, surf_n: int, surf_dx: float,
                      shift=(0.0, 0.0), rotation: float = 0.0, magnification: float = 1.0) -> np.ndarray:
    """Surface of a translated, rotated and magnified DM by the direct sum over actuators."""
    C_ = np.ascontiguousarray(cmd_grid, dtype=np.float64)
    out = np.zeros((surf_n, surf_n))
    lib().orc_dm_surface_misreg(C_.shape[1], C_.shape[0], pitch, coupling, surf_n, surf_dx, shift[0], shift[1],
                                rotation, magnification, _ptr(C_, C.c_double), _ptr(out, C.c_double))
    return out


def bin_image(img: np.ndarray, n_bin: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.float64)
    n = img.shape[0]
    out = np.zeros((n // n_bin, n // n_bin))
    lib().orc_bin(n, n_bin, _ptr(img, C.c_double), _ptr(out, C.c_double))
    return out


def cog(img: np.ndarray):
    img = np.ascontiguousarray(img, dtype=np.float64)
    sx, sy = C.c_double(), C.c_double()
    lib().orc_cog(img.shape[0], _ptr(img, C.c_double), C.byref(sx), C.byref(sy))
    return sx.value, sy.value


def subap_slopes(amp: np.ndarray, phase: np.ndarray, n_fft: int, n_bin: int, sigma_pix: float = 0.0,
                 direction=(1.0, 0.0)):
    """Noise-free centre-of-gravity slopes of one subaperture: cog(bin(sh_image)) (phase in rad
    at the sensing wavelength); the flux normalisation does not change a centroid."""
    return cog(bin_image(sh_image(amp, phase, n_fft, sigma_pix, direction), n_bin))


def subap_jacobian_fd(amp: np.ndarray, phase: np.ndarray, n_fft: int, n_bin: int, sigma_pix: float = 0.0,
                      direction=(1.0, 0.0), h: float = 1e-4) -> np.ndarray:
    """d (sx, sy) / d phase of one subaperture by central differences of subap_slopes (the
    derivative's definition; truncation O(h^2)): [2][n_px][n_px]."""
    phase = np.array(phase, dtype=np.float64)
    out = np.zeros((2,) + phase.shape)
    for j in range(phase.shape[0]):
        for i in range(phase.shape[1]):
            p = phase.copy()
            p[j, i] += h
            sp = subap_slopes(amp, p, n_fft, n_bin, sigma_pix, direction)
            p[j, i] -= 2 * h
            sm = subap_slopes(amp, p, n_fft, n_bin, sigma_pix, direction)
            out[0, j, i] = (sp[0] - sm[0]) / (2 * h)
            out[1, j, i] = (sp[1] - sm[1]) / (2 * h)
    return out


def jacobian_fd(sim: "Sim", h: float = 1e-3) -> np.ndarray:
    """Interaction matrix d slopes / d commands at the simulation's current step and commands by
    central differences of its measurement (the derivative's definition, truncation O(h^2));
    the configuration must be noise-free.  Restores the commands."""
    c0 = sim.commands().copy()
    D = np.zeros((sim.n_slopes, sim.n_cmd))
    for j in range(sim.n_cmd):
        c = c0.copy()
        c[j] += h
        sim.set_commands(c)
        sp = sim.measure()
        c[j] = c0[j] - h
        sim.set_commands(c)
        D[:, j] = (sp - sim.measure()) / (2 * h)
    sim.set_commands(c0)
    return D


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(o, C.c_uint32))
    return o


def uniform_f32(w: int) -> float:
    return lib().orc_uniform_f32(int(w) & 0xFFFFFFFF)


def exp_f32(x: float) -> float:
    return lib().orc_exp_f32(x)


def log_f32(x: float) -> float:
    return lib().orc_log_f32(x)


def sincos2pi_f32(x: float):
    """(cos 2 pi x, sin 2 pi x) of the sampler's float polynomials."""
    c, s = C.c_float(), C.c_float()
    lib().orc_sincos2pi_f32(x, C.byref(c), C.byref(s))
    return c.value, s.value


def bf16_rn(x: float) -> int:
    return lib().orc_bf16_rn(x)


def bf16_to_f32(h: int) -> float:
    return lib().orc_bf16_to_f32(h)


def e4m3_rn_sat(x: float) -> int:
    return lib().orc_e4m3_rn_sat(x)


def e4m3_to_f32(b: int) -> float:
    return lib().orc_e4m3_to_f32(b)


def quantize_rows(R: np.ndarray, dtype: int):
    """(codes, scales) of the rows of R: bfloat16 codes (uint16) with scale 1, or FP8 E4M3 codes
    (uint8) with one float scale per row."""
    R = np.ascontiguousarray(R, dtype=np.float32)
    rows, cols = R.shape
    out = np.empty((rows, cols), np.uint16 if dtype == DTYPE_BF16 else np.uint8)
    sc = np.empty(rows, np.float32)
    lib().orc_quantize_rows(_ptr(R, C.c_float), rows, cols, cols, dtype, out.ctypes.data, _ptr(sc, C.c_float))
    return out, sc


def dequantize_rows(codes: np.ndarray, scales: np.ndarray, dtype: int) -> np.ndarray:
    """float64 values represented by the codes (the definition the reduced-precision product uses)."""
    if dtype == DTYPE_BF16:
        return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    table = np.array([e4m3_to_f32(b) for b in range(256)], dtype=np.float64)
    return table[codes] * scales.astype(np.float64)[:, None]


def noise_pair(lam_a: float, lam_b: float, read_noise: float, c0: int, c1: int, c2: int, seed: int):
    """Noisy counts of a pixel pair (see orc_noise_pair)."""
    a, b = C.c_int32(), C.c_int32()
    lib().orc_noise_pair(lam_a, lam_b, read_noise, c0, c1, c2, seed, C.byref(a), C.byref(b))
    return a.value, b.value


def noise_frame(lam: np.ndarray, read_noise: float, pixel0: int, step: int, wfs: int, seed: int,
                frame_px: int) -> np.ndarray:
    """Noisy frames of a buffer of subaperture frames of frame_px pixels (pairs within frames)."""
    lam = np.ascontiguousarray(lam, dtype=np.float32).ravel()
    out = np.zeros(lam.size, dtype=np.int32)
    lib().orc_noise_frame(_ptr(lam, C.c_float), lam.size, int(frame_px), read_noise, pixel0, step, wfs, seed,
                          _ptr(out, C.c_int32))
    return out


def screen_coeffs(n: int, pixel: float, r0: float, L0: float, seed: int) -> np.ndarray:
    """Complex coefficients c_k of the FFT-method phase screen, [ky][kx] (see orc_screen_coeffs)."""
    re = np.zeros((n, n))
    im = np.zeros((n, n))
    lib().orc_screen_coeffs(int(n), float(pixel), float(r0), float(L0), int(seed) & 0xFFFFFFFFFFFFFFFF,
                            _ptr(re, C.c_double), _ptr(im, C.c_double))
    return re + 1j * im


def phase_screen(n: int, pixel: float, r0: float, L0: float, seed: int) -> np.ndarray:
    """Von Karman phase screen by the FFT method ("The atmospheric layers generation"):
    Re sum_k c_k exp(2 pi i k.x / n), i.e. n^2 times the inverse DFT of the coefficients;
    [y][x] in rad."""
    return np.real(np.fft.ifft2(screen_coeffs(n, pixel, r0, L0, seed))) * (n * n)


def screen_amp(n: int, pixel: float, r0: float, L0: float) -> np.ndarray:
    """Amplitudes a_k of the FFT-method screen coefficients, [ky][kx] (see orc_screen_amp)."""
    a = np.zeros((n, n))
    lib().orc_screen_amp(int(n), float(pixel), float(r0), float(L0), _ptr(a, C.c_double))
    return a


def screen_structure_function(n: int, pixel: float, r0: float, L0: float, r_px: int) -> float:
    """Expected structure function of the FFT-method screen at a lag of r_px samples along x:
    E (phi(x + r) - phi(x))^2 = sum_k a_k^2 2 (1 - cos(2 pi kx r / n)) (each term
    Re(c_k e^{i t}) has variance a_k^2, the terms are independent)."""
    a2 = screen_amp(n, pixel, r0, L0) ** 2
    kx = np.arange(n)[None, :]
    return float(np.sum(a2 * 2.0 * (1.0 - np.cos(2 * np.pi * kx * r_px / n))))


def tikhonov_reconstructor(D: np.ndarray, alpha: float):
    """Control matrix by Tikhonov-regularised least squares ("Control Matrix": the reconstructor is
    a regularised pseudo-inverse of the interaction matrix, MCAO least squares being ill-posed):
    R = -(D^T D + lam I)^-1 D^T with lam = alpha tr(D^T D) / n_cmd (reading: the regularisation
    weight is relative to the mean eigenvalue of D^T D), in double, the normal equations solved by
    LAPACK (numpy.linalg.solve).  The minus sign: D is measured with the DM subtracted from the
    wavefront and the loop adds g R s to the commands.  D is [n_slopes][n_cmd]; returns (R, lam),
    R [n_cmd][n_slopes]."""
    D = np.asarray(D, dtype=np.float64)
    G = D.T @ D
    lam = alpha * np.trace(G) / G.shape[0]
    return -np.linalg.solve(G + lam * np.eye(G.shape[0]), D.T), lam


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------------------------------------
# whole simulation
# ------------------------------------------------------------------------------------------

class Sim:
    """Closed-loop simulation state of the oracle for one configuration dictionary."""

    def __init__(self, cfg: dict, screens, R: np.ndarray | None = None, s_ref: np.ndarray | None = None,
                 r_dtype: int = DTYPE_F32):
        L = lib()
        self._keep = []
        nw, ns, nl, nd = len(cfg["wfs"]), len(cfg["science"]), len(cfg["layers"]), len(cfg["dms"])
        wfs = (_Wfs * max(nw, 1))()
        for i, w in enumerate(cfg["wfs"]):
            wfs[i] = _Wfs(1 if w["type"] == "lgs" else 0, w["n_sub"], w["n_px"], w["n_fft"], w["n_bin"], 0,
                          w["theta"][0], w["theta"][1], w["height"], w["lambda"], w["n_photons"],
                          w["read_noise"], w["valid_thr"], w["na_fwhm"], w["launch"][0], w["launch"][1])
        sci = (_Sci * max(ns, 1))()
        for i, s in enumerate(cfg["science"]):
            sci[i] = _Sci(s["n_px"], s["pad"], s["theta"][0], s["theta"][1], s["lambda"])
        lay = (_Layer * max(nl, 1))()
        for i, (l, scr) in enumerate(zip(cfg["layers"], screens)):
            a = np.ascontiguousarray(scr, dtype=np.float32)
            self._keep.append(a)
            lay[i] = _Layer(l["n"], 0, l["pixel"], l["alt"], l["vx"], l["vy"], _ptr(a, C.c_float))
        dms = (_Dm * max(nd, 1))()
        for i, d in enumerate(cfg["dms"]):
            v = np.ascontiguousarray(d["valid"], dtype=np.uint8)
            self._keep.append(v)
            dms[i] = _Dm(d["nx"], d["ny"], d["surf_n"], 0, d["alt"], d["pitch"], d["coupling"],
                         d["surf_dx"], _ptr(v, C.c_uint8))
        c = _Config()
        c.D, c.obstruction, c.lambda_ref = cfg["D"], cfg["obstruction"], cfg["lambda_ref"]
        c.dt, c.gain, c.seed = cfg["dt"], cfg["gain"], cfg["seed"]
        c.noise, c.psf_every = int(cfg["noise"]), int(cfg.get("psf_every", 1))
        c.n_wfs, c.n_sci, c.n_layers, c.n_dms = nw, ns, nl, nd
        c.wfs, c.sci, c.layers, c.dms = wfs, sci, lay, dms
        if R is not None:
            R = np.ascontiguousarray(R, dtype=np.float32)
            self._keep.append(R)
            c.n_cmd, c.n_slopes = R.shape
            c.R = _ptr(R, C.c_float)
        if s_ref is not None:
            s_ref = np.ascontiguousarray(s_ref, dtype=np.float32)
            self._keep.append(s_ref)
            c.s_ref = _ptr(s_ref, C.c_float)
        c.r_dtype = int(r_dtype)
        self._cfg_struct = (c, wfs, sci, lay, dms)
        self.h = L.orc_create(C.byref(c))
        if not self.h:
            raise ValueError("oracle rejected the configuration (reconstructor shape mismatch?)")
        self.cfg = cfg
        self.n_cmd = L.orc_n_cmd(self.h)
        self.n_slopes = L.orc_n_slopes(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1):
        if lib().orc_step(self.h, n) != 0:
            raise RuntimeError("oracle step needs a reconstructor")

    def measure(self) -> np.ndarray:
        out = np.zeros(self.n_slopes)
        lib().orc_measure(self.h, _ptr(out, C.c_double))
        return out

    @property
    def k(self) -> int:
        return lib().orc_step_index(self.h)

    @k.setter
    def k(self, v: int):
        lib().orc_set_step_index(self.h, int(v))

    def n_valid(self, w: int) -> int:
        return lib().orc_n_valid(self.h, w)

    def valid(self, w: int) -> np.ndarray:
        out = np.zeros(self.n_valid(w), dtype=np.int32)
        lib().orc_get_valid(self.h, w, _ptr(out, C.c_int))
        return out

    def slopes(self) -> np.ndarray:
        out = np.zeros(self.n_slopes)
        lib().orc_get_slopes(self.h, _ptr(out, C.c_double))
        return out

    def commands(self) -> np.ndarray:
        out = np.zeros(self.n_cmd)
        lib().orc_get_commands(self.h, _ptr(out, C.c_double))
        return out

    def set_commands(self, c: np.ndarray):
        c = np.ascontiguousarray(c, dtype=np.float64)
        assert c.size == self.n_cmd
        lib().orc_set_commands(self.h, _ptr(c, C.c_double))

    def set_sodium(self, w: int, height: float, na_fwhm: float):
        """Sodium layer height and thickness seen by laser sensor w from the next step on."""
        if lib().orc_set_sodium(self.h, w, height, na_fwhm) != 0:
            raise ValueError("not a laser sensor, or height not above every layer")

    def marechal(self, q: int = 0):
        """(long-exposure, last-step) Marechal Strehl of science direction q."""
        a, b = C.c_double(), C.c_double()
        lib().orc_marechal(self.h, q, C.byref(a), C.byref(b))
        return a.value, b.value

    def set_controller(self, a1: float, a2: float, b0: float, b1: float):
        """Second-order controller c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1}."""
        lib().orc_set_controller(self.h, a1, a2, b0, b1)

    def dm_surface(self, m: int) -> np.ndarray:
        n = self.cfg["dms"][m]["surf_n"]
        out = np.zeros((n, n))
        lib().orc_get_dm_surface(self.h, m, _ptr(out, C.c_double))
        return out

    def set_misregistration(self, m: int, shift_x: float, shift_y: float, rotation: float, magnification: float):
        """DM m seen through T(q) = magnification R(rotation) q + shift (m, rad) from the next
        measurement on."""
        if lib().orc_set_misregistration(self.h, m, shift_x, shift_y, rotation, magnification) != 0:
            raise ValueError("bad DM index or magnification")

    def elongation(self, w: int):
        """(sigma in image pixels [n_valid], unit direction [n_valid][2]) of sensor w's spots."""
        nv = lib().orc_n_valid(self.h, w)
        sig = np.zeros(nv)
        d = np.zeros((nv, 2))
        lib().orc_get_elongation(self.h, w, _ptr(sig, C.c_double), _ptr(d, C.c_double))
        return sig, d

    def wfs_phase(self, w: int) -> np.ndarray:
        ww = self.cfg["wfs"][w]
        n = ww["n_sub"] * ww["n_px"]
        out = np.zeros((n, n))
        lib().orc_wfs_phase(self.h, w, _ptr(out, C.c_double))
        return out

    def frames(self, w: int):
        ww = self.cfg["wfs"][w]
        nd = ww["n_fft"] // ww["n_bin"]
        nv = self.n_valid(w)
        lam = np.zeros((nv, nd, nd), dtype=np.float32)
        fr = np.zeros((nv, nd, nd), dtype=np.int32)
        lib().orc_get_frames(self.h, w, _ptr(lam, C.c_float), _ptr(fr, C.c_int32))
        return lam, fr

    def psf(self, q: int = 0):
        s = self.cfg["science"][q]
        M = s["n_px"] * s["pad"]
        out = np.zeros((M, M))
        srl, srk = C.c_double(), C.c_double()
        lib().orc_get_psf(self.h, q, _ptr(out, C.c_double), C.byref(srl), C.byref(srk))
        return out, srl.value, srk.value
