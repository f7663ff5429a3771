"""Thin ctypes binding of libmcao.so (include/mcao.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Arrays may be numpy arrays (host) or
CUDA torch tensors (device, passed by address with ``on_device = 1`` where the ABI allows it).
If the library has not been built, or no CUDA device is available, the calls raise: there is
no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

STATUS = {0: "MCAO_OK", 1: "MCAO_E_INVALID_ARG", 2: "MCAO_E_SHAPE", 3: "MCAO_E_STATE", 4: "MCAO_E_CUDA",
          5: "MCAO_E_OOM", 6: "MCAO_E_TIMEOUT", 7: "MCAO_E_UNSUPPORTED"}
Q_SLOPES, Q_COMMANDS, Q_VALID, Q_FRAME, Q_WFS_PHASE, Q_DM_SURFACE, Q_PSF, Q_STATE, Q_REALIZATIONS = range(9)
STAGES = ["dm", "wfs_main", "wfs_aux", "recon", "recon_reduce", "science"]

# exported names of include/mcao.h (checked by the tests against the built library)
EXPORTS = [
    "mcao_sim_create", "mcao_sim_destroy", "mcao_last_error", "mcao_create_error", "mcao_set_stream",
    "mcao_load_atmosphere", "mcao_load_dms", "mcao_load_reconstructor", "mcao_step", "mcao_sync",
    "mcao_query", "mcao_get_step_index", "mcao_get_slopes", "mcao_get_commands", "mcao_set_commands",
    "mcao_get_valid", "mcao_get_wfs_phase", "mcao_get_dm_surface", "mcao_get_frames", "mcao_get_psf",
    "mcao_reset_psf", "mcao_get_state", "mcao_set_state", "mcao_set_profiling", "mcao_set_profiling_stages", "mcao_get_profile",
    "mcao_reconstruct_noalloc", "mcao_get_timeline", "mcao_quantize_rows", "mcao_set_realization",
    "mcao_set_controller", "mcao_get_marechal", "mcao_set_sodium", "mcao_generate_screen", "mcao_measure",
    "mcao_interaction_matrix", "mcao_slopes_vjp", "mcao_set_misregistration", "mcao_step_group",
    "mcao_read_async", "mcao_check_bounded_wait", "mcao_reconstruct_batch", "mcao_tikhonov_reconstructor",
    "mcao_misreg_normal_equations", "mcao_get_tuning", "mcao_set_tuning", "mcao_autotune",
]

DTYPE_F32, DTYPE_BF16, DTYPE_FP8_E4M3 = 0, 1, 2


class McaoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Wfs(C.Structure):
    _fields_ = [("type", C.c_int), ("n_sub", C.c_int), ("n_px", C.c_int), ("n_fft", C.c_int), ("n_bin", C.c_int),
                ("theta_x", C.c_double), ("theta_y", C.c_double), ("height", C.c_double), ("lambda_", C.c_double),
                ("n_photons", C.c_double), ("read_noise", C.c_double), ("valid_thr", C.c_double),
                ("na_fwhm", C.c_double), ("launch_x", C.c_double), ("launch_y", C.c_double)]


class _Science(C.Structure):
    _fields_ = [("n_px", C.c_int), ("pad", C.c_int), ("theta_x", C.c_double), ("theta_y", C.c_double),
                ("lambda_", C.c_double)]


class _Config(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("D", C.c_double), ("obstruction", C.c_double),
                ("lambda_ref", C.c_double), ("dt", C.c_double), ("gain", C.c_double), ("seed", C.c_uint64),
                ("noise", C.c_int), ("psf_every", C.c_int), ("keep_frames", C.c_int), ("n_wfs", C.c_int),
                ("wfs", C.POINTER(_Wfs)), ("n_sci", C.c_int), ("sci", C.POINTER(_Science)), ("n_real", C.c_int)]


class _Layer(C.Structure):
    _fields_ = [("n", C.c_int), ("pixel_m", C.c_double), ("alt_m", C.c_double), ("vx", C.c_double),
                ("vy", C.c_double), ("phase", C.c_void_p), ("on_device", C.c_int)]


class _Dm(C.Structure):
    _fields_ = [("alt_m", C.c_double), ("pitch_m", C.c_double), ("coupling", C.c_double), ("nx", C.c_int),
                ("ny", C.c_int), ("valid", C.POINTER(C.c_uint8)), ("surf_n", C.c_int), ("surf_dx", C.c_double)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmcao.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (paper_1608_00386_gb300.build.build())")
    L = C.CDLL(path)
    vp, st = C.c_void_p, C.c_int
    sig = {
        "mcao_sim_create": [C.POINTER(_Config), C.POINTER(vp)],
        "mcao_sim_destroy": [vp],
        "mcao_set_stream": [vp, vp],
        "mcao_load_atmosphere": [vp, C.c_int, C.POINTER(_Layer)],
        "mcao_load_dms": [vp, C.c_int, C.POINTER(_Dm)],
        "mcao_load_reconstructor": [vp, C.c_int, C.c_int, vp, vp, C.c_int, C.c_int],
        "mcao_step": [vp, C.c_int],
        "mcao_sync": [vp],
        "mcao_query": [vp, C.c_int, C.c_int, C.POINTER(C.c_size_t)],
        "mcao_get_step_index": [vp, C.POINTER(C.c_int64)],
        "mcao_get_slopes": [vp, vp, C.c_size_t],
        "mcao_get_commands": [vp, vp, C.c_size_t],
        "mcao_set_commands": [vp, vp, C.c_size_t],
        "mcao_get_valid": [vp, C.c_int, vp, C.c_size_t],
        "mcao_get_wfs_phase": [vp, C.c_int, vp, C.c_size_t],
        "mcao_get_dm_surface": [vp, C.c_int, vp, C.c_size_t],
        "mcao_get_frames": [vp, C.c_int, vp, vp, C.c_size_t],
        "mcao_get_psf": [vp, C.c_int, vp, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "mcao_reset_psf": [vp],
        "mcao_get_state": [vp, vp, C.c_size_t],
        "mcao_set_state": [vp, vp, C.c_size_t],
        "mcao_set_profiling": [vp, C.c_int],
        "mcao_set_profiling_stages": [vp, C.c_uint],
        "mcao_get_profile": [vp, vp, vp, C.c_int, C.POINTER(C.c_int64)],
        "mcao_reconstruct_noalloc": [vp, C.c_int, C.c_int, C.c_int, vp, vp, C.c_float, vp, C.c_char_p, C.c_size_t],
        "mcao_get_timeline": [vp, vp, vp, vp, vp, C.c_size_t, C.POINTER(C.c_size_t)],
        "mcao_quantize_rows": [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_char_p, C.c_size_t],
        "mcao_set_realization": [vp, C.c_int],
        "mcao_set_controller": [vp, C.c_double, C.c_double, C.c_double, C.c_double],
        "mcao_get_marechal": [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "mcao_set_sodium": [vp, C.c_int, C.c_double, C.c_double],
        "mcao_generate_screen": [C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64, vp, vp, C.c_char_p,
                                 C.c_size_t],
        "mcao_measure": [vp, C.c_int],
        "mcao_interaction_matrix": [vp, vp, C.c_size_t],
        "mcao_slopes_vjp": [vp, vp, C.c_int, vp, vp, vp],
        "mcao_set_misregistration": [vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double],
        "mcao_step_group": [C.POINTER(vp), C.c_int, C.c_int],
        "mcao_read_async": [vp, vp, vp],
        "mcao_check_bounded_wait": [vp],
        "mcao_reconstruct_batch": [vp, vp, C.c_int, vp],
        "mcao_tikhonov_reconstructor": [vp, C.c_int, C.c_int, C.c_size_t, C.c_double, vp, C.c_size_t, C.c_int, vp,
                                        C.POINTER(C.c_double), C.c_char_p, C.c_size_t],
        "mcao_misreg_normal_equations": [vp, C.c_int, vp, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "mcao_get_tuning": [vp, C.POINTER(C.c_int), C.c_int],
        "mcao_set_tuning": [vp, C.POINTER(C.c_int), C.c_int],
        "mcao_autotune": [vp, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_char_p, C.c_size_t],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.mcao_last_error.argtypes = [vp]
    L.mcao_last_error.restype = C.c_char_p
    L.mcao_create_error.argtypes = []
    L.mcao_create_error.restype = C.c_char_p
    _lib = L
    return L


def _addr(a):
    """(address, keepalive, on_device) of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), a, int(a.is_cuda)
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a, 0


class Sim:
    """One closed-loop simulation handle (mcao_sim)."""

    def __init__(self, cfg: dict, keep_frames: bool = False, stream=None, n_real: int = 1):
        L = lib()
        self.cfg = cfg
        nw, nsci = len(cfg["wfs"]), len(cfg["science"])
        self._wfs = (_Wfs * nw)()
        for i, w in enumerate(cfg["wfs"]):
            self._wfs[i] = _Wfs(1 if w["type"] == "lgs" else 0, w["n_sub"], w["n_px"], w["n_fft"], w["n_bin"],
                                w["theta"][0], w["theta"][1], w["height"], w["lambda"], w["n_photons"],
                                w["read_noise"], w["valid_thr"], w["na_fwhm"], w["launch"][0], w["launch"][1])
        self._sci = (_Science * max(nsci, 1))()
        for i, s in enumerate(cfg["science"]):
            self._sci[i] = _Science(s["n_px"], s["pad"], s["theta"][0], s["theta"][1], s["lambda"])
        c = _Config()
        c.struct_size = C.sizeof(_Config)
        c.D, c.obstruction, c.lambda_ref = cfg["D"], cfg["obstruction"], cfg["lambda_ref"]
        c.dt, c.gain, c.seed = cfg["dt"], cfg["gain"], cfg["seed"]
        c.noise, c.psf_every, c.keep_frames = int(cfg["noise"]), int(cfg.get("psf_every", 1)), int(keep_frames)
        c.n_wfs, c.wfs, c.n_sci, c.sci = nw, self._wfs, nsci, self._sci
        c.n_real = int(n_real)
        self.n_real = int(n_real)
        h = C.c_void_p()
        st = L.mcao_sim_create(C.byref(c), C.byref(h))
        if st != 0:
            raise McaoError(st, L.mcao_create_error().decode())
        self.h = h
        self._keep = []
        if stream is not None:
            self.set_stream(stream)

    # ---------------------------------------------------------------- plumbing
    def _ck(self, st):
        if st != 0:
            raise McaoError(st, lib().mcao_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().mcao_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, kind: int, index: int = 0) -> int:
        n = C.c_size_t()
        self._ck(lib().mcao_query(self.h, kind, index, C.byref(n)))
        return n.value

    def set_stream(self, stream):
        ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._ck(lib().mcao_set_stream(self.h, C.c_void_p(ptr)))

    # ---------------------------------------------------------------- loads
    def set_sodium(self, w: int, height: float, na_fwhm: float):
        """Sodium layer height and thickness seen by laser sensor w from the next step on."""
        self._ck(lib().mcao_set_sodium(self.h, int(w), float(height), float(na_fwhm)))

    def marechal(self, q: int = 0):
        """(long-exposure, last-step) Marechal Strehl of science direction q."""
        a, b = C.c_double(), C.c_double()
        self._ck(lib().mcao_get_marechal(self.h, int(q), C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_controller(self, a1: float, a2: float, b0: float, b1: float):
        """Second-order controller c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1}."""
        self._ck(lib().mcao_set_controller(self.h, float(a1), float(a2), float(b0), float(b1)))

    def set_realization(self, r: int):
        """Address realization r in later loads of screens, getters and command setters."""
        self._ck(lib().mcao_set_realization(self.h, int(r)))

    def load_atmosphere(self, screens, realization: int | None = None):
        if realization is not None:
            self.set_realization(realization)
        layers = (_Layer * len(screens))()
        keep = []
        for i, (lay, scr) in enumerate(zip(self.cfg["layers"], screens)):
            if not hasattr(scr, "data_ptr"):
                scr = np.ascontiguousarray(scr, dtype=np.float32)
            addr, k, dev = _addr(scr)
            keep.append(k)
            layers[i] = _Layer(lay["n"], lay["pixel"], lay["alt"], lay["vx"], lay["vy"], addr, dev)
        self._ck(lib().mcao_load_atmosphere(self.h, len(screens), layers))
        self._keep.append(keep)  # device tensors are adopted: keep them alive

    def generate_atmosphere(self, realization: int | None = None, seed_offset: int = 0):
        """Generate every layer's screen on the device (mcao_generate_screen with the layer's n,
        pixel, r0, L0 and seed + seed_offset) and load them for the selected realization."""
        scr = [generate_screen(lay["n"], lay["pixel"], lay["r0"], lay["L0"], lay["seed"] + seed_offset)
               for lay in self.cfg["layers"]]
        import torch
        torch.cuda.current_stream().synchronize()   # the simulation's streams do not wait on torch's
        self.load_atmosphere(scr, realization)
        return scr

    def load_dms(self):
        dms = self.cfg["dms"]
        arr = (_Dm * max(len(dms), 1))()
        keep = []
        for i, d in enumerate(dms):
            v = np.ascontiguousarray(d["valid"], dtype=np.uint8)
            keep.append(v)
            arr[i] = _Dm(d["alt"], d["pitch"], d["coupling"], d["nx"], d["ny"],
                         v.ctypes.data_as(C.POINTER(C.c_uint8)), d["surf_n"], d["surf_dx"])
        self._ck(lib().mcao_load_dms(self.h, len(dms), arr))

    def load_reconstructor(self, R, s_ref=None, dtype: int = DTYPE_F32):
        if not hasattr(R, "data_ptr"):
            R = np.ascontiguousarray(R, dtype=np.float32)
        addr, k, dev = _addr(R)
        sp = None
        if s_ref is not None:
            if not hasattr(s_ref, "data_ptr"):
                s_ref = np.ascontiguousarray(s_ref, dtype=np.float32)
            sp, ks, sdev = _addr(s_ref)
            if sdev != dev:
                raise ValueError("R and s_ref must both be on the host or both on the device")
        self._ck(lib().mcao_load_reconstructor(self.h, R.shape[0], R.shape[1], addr, sp, int(dtype), dev))

    # ---------------------------------------------------------------- loop
    def step(self, n: int = 1):
        self._ck(lib().mcao_step(self.h, int(n)))

    def sync(self):
        self._ck(lib().mcao_sync(self.h))

    @property
    def step_index(self) -> int:
        k = C.c_int64()
        self._ck(lib().mcao_get_step_index(self.h, C.byref(k)))
        return k.value

    # ---------------------------------------------------------------- outputs
    def slopes(self, out=None) -> np.ndarray:
        n = self.query(Q_SLOPES)
        out = np.empty(n, np.float32) if out is None else out
        self._ck(lib().mcao_get_slopes(self.h, out.ctypes.data, out.size))
        return out

    def commands(self, out=None) -> np.ndarray:
        n = self.query(Q_COMMANDS)
        out = np.empty(n, np.float32) if out is None else out
        self._ck(lib().mcao_get_commands(self.h, out.ctypes.data, out.size))
        return out

    def set_commands(self, c):
        c = np.ascontiguousarray(c, dtype=np.float32)
        self._ck(lib().mcao_set_commands(self.h, c.ctypes.data, c.size))

    def set_misregistration(self, dm: int, shift_x: float = 0.0, shift_y: float = 0.0, rotation: float = 0.0,
                            magnification: float = 1.0):
        """Move DM dm as a rigid body (shift in m, rotation in rad, magnification)."""
        self._ck(lib().mcao_set_misregistration(self.h, dm, shift_x, shift_y, rotation, magnification))

    def reconstruct_batch(self, S):
        """R s_r for every row s_r of the CUDA float32 tensor S [n_rhs][n_slopes] with the loaded
        control matrix, by the batched step's product kernels (mcao_reconstruct_batch); returns a
        CUDA float32 tensor [n_rhs][n_commands]."""
        import torch
        if not (isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.float32 and S.dim() == 2
                and S.is_contiguous() and S.shape[1] == self.query(Q_SLOPES)):
            raise McaoError(1, "S must be a contiguous CUDA float32 tensor [n_rhs][n_slopes]")
        out = torch.empty((S.shape[0], self.query(Q_COMMANDS)), dtype=torch.float32, device=S.device)
        self._ck(lib().mcao_reconstruct_batch(self.h, S.data_ptr(), S.shape[0], out.data_ptr()))
        return out

    def misreg_normal_equations(self, dm: int, D_meas):
        """Gauss-Newton terms of DM dm's misregistration fit at its current misregistration
        (mcao_misreg_normal_equations): D_meas is a CUDA float32 tensor [n_slopes][>= the DM's
        commands] with unit column stride whose column j is the DM's command j.  Returns (JtJ
        [4][4], Jte [4], cost, meas_sq) as numpy / floats."""
        import torch
        if not (isinstance(D_meas, torch.Tensor) and D_meas.is_cuda and D_meas.dtype == torch.float32
                and D_meas.dim() == 2 and D_meas.stride(1) == 1 and D_meas.shape[0] == self.query(Q_SLOPES)):
            raise McaoError(1, "D_meas must be a CUDA float32 tensor [n_slopes][n] with unit column stride")
        JtJ = (C.c_double * 16)()
        Jte = (C.c_double * 4)()
        cost, msq = C.c_double(), C.c_double()
        self._ck(lib().mcao_misreg_normal_equations(self.h, int(dm), D_meas.data_ptr(), D_meas.stride(0), JtJ, Jte,
                                                    C.byref(cost), C.byref(msq)))
        return np.array(JtJ[:]).reshape(4, 4), np.array(Jte[:]), cost.value, msq.value

    TUNING = ("sense_blocks_per_sm", "recon_ctas_pct", "science_after_aux", "tc_chunk", "multi_blocks_per_sm",
              "steps_per_graph")

    def tuning(self) -> dict:
        """Current launch shapes (mcao_get_tuning), by name."""
        v = (C.c_int * len(self.TUNING))()
        self._ck(lib().mcao_get_tuning(self.h, v, len(self.TUNING)))
        return dict(zip(self.TUNING, v[:]))

    def set_tuning(self, **kw):
        """Change launch shapes by name (mcao_set_tuning); the others keep their values."""
        cur = self.tuning()
        for k, val in kw.items():
            if k not in cur:
                raise McaoError(1, f"unknown tuning knob {k}")
            cur[k] = int(val)
        v = (C.c_int * len(self.TUNING))(*[cur[k] for k in self.TUNING])
        self._ck(lib().mcao_set_tuning(self.h, v, len(self.TUNING)))

    def autotune(self, steps_per_trial: int = 50):
        """Time every candidate launch shape of this configuration and keep the fastest
        (mcao_autotune); the simulation's state is restored afterwards.  Returns (chosen shapes by
        name, report string)."""
        v = (C.c_int * len(self.TUNING))()
        buf = C.create_string_buffer(4096)
        self._ck(lib().mcao_autotune(self.h, int(steps_per_trial), v, len(self.TUNING), buf, 4096))
        return dict(zip(self.TUNING, v[:])), buf.value.decode()

    def check_bounded_wait(self) -> int:
        """Status of mcao_check_bounded_wait: 6 (MCAO_E_TIMEOUT) when the device timeouts work."""
        return lib().mcao_check_bounded_wait(self.h)

    def read_async(self, commands=None, strehl=None):
        """Queue copies of the commands (float32 [n_commands]) and the (long, last) Strehl ratios
        (float64 [n_sci][2]) into the given host arrays (pinned: torch tensors with
        pin_memory(), or numpy views of them) after the queued work; valid after sync()."""
        ptr = lambda a: (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data) if a is not None else None
        self._ck(lib().mcao_read_async(self.h, ptr(commands), ptr(strehl)))

    def measure(self, noise: bool = False) -> np.ndarray:
        """Slopes at the current step and commands without reconstruction or time advance
        (noise-free unless noise=True and the configuration has noise)."""
        self._ck(lib().mcao_measure(self.h, int(bool(noise))))
        return self.slopes()

    def interaction_matrix(self):
        """Exact Jacobian d slopes / d commands of the noise-free slopes at the current state, as a
        CUDA float32 tensor [n_slopes][n_commands] (mcao_interaction_matrix)."""
        import torch
        D = torch.empty((self.query(Q_SLOPES), self.query(Q_COMMANDS)), dtype=torch.float32, device="cuda")
        self._ck(lib().mcao_interaction_matrix(self.h, D.data_ptr(), D.shape[1]))
        return D

    def slopes_vjp(self, g, commands: bool = True, phase: bool = False, layers: bool = False):
        """Vector-Jacobian products of the noise-free slopes (mcao_slopes_vjp) for g, a CUDA tensor
        [n_slopes] or [n_vec][n_slopes]: command gradients [.., n_commands], pupil-phase gradients
        [.., sum of N_w^2] and layer gradients [.., sum of n_l^2] (each None unless asked), shaped
        like g; with layers=True a third element is returned."""
        import torch
        ns, nc = self.query(Q_SLOPES), self.query(Q_COMMANDS)
        g2 = g.detach().to(device="cuda", dtype=torch.float32).reshape(-1, ns).contiguous()
        nv = g2.shape[0]
        gc = torch.empty((nv, nc), dtype=torch.float32, device="cuda") if commands else None
        nph = sum(self.query(Q_WFS_PHASE, w) for w in range(len(self.cfg["wfs"])))
        gp = torch.empty((nv, nph), dtype=torch.float32, device="cuda") if phase else None
        nly = sum(l["n"] ** 2 for l in self.cfg["layers"])
        gl = torch.empty((nv, nly), dtype=torch.float32, device="cuda") if layers else None
        ptr = lambda t: t.data_ptr() if t is not None else None
        self._ck(lib().mcao_slopes_vjp(self.h, g2.data_ptr(), nv, ptr(gc), ptr(gp), ptr(gl)))
        if g.dim() == 1:
            gc, gp, gl = [t[0] if t is not None else None for t in (gc, gp, gl)]
        return (gc, gp, gl) if layers else (gc, gp)

    def valid(self, w: int) -> np.ndarray:
        out = np.empty(self.query(Q_VALID, w), np.int32)
        self._ck(lib().mcao_get_valid(self.h, w, out.ctypes.data, out.size))
        return out

    def wfs_phase(self, w: int) -> np.ndarray:
        ww = self.cfg["wfs"][w]
        n = ww["n_sub"] * ww["n_px"]
        out = np.empty((n, n), np.float32)
        self._ck(lib().mcao_get_wfs_phase(self.h, w, out.ctypes.data, out.size))
        return out

    def dm_surface(self, m: int) -> np.ndarray:
        n = self.cfg["dms"][m]["surf_n"]
        out = np.empty((n, n), np.float32)
        self._ck(lib().mcao_get_dm_surface(self.h, m, out.ctypes.data, out.size))
        return out

    def frames(self, w: int):
        ww = self.cfg["wfs"][w]
        nd = ww["n_fft"] // ww["n_bin"]
        nv = self.query(Q_VALID, w)
        lam = np.empty((nv, nd, nd), np.float32)
        fr = np.empty((nv, nd, nd), np.int32)
        self._ck(lib().mcao_get_frames(self.h, w, lam.ctypes.data, fr.ctypes.data, lam.size))
        return lam, fr

    def psf(self, q: int = 0, with_image: bool = True):
        M = self.cfg["science"][q]["n_px"] * self.cfg["science"][q]["pad"]
        out = np.empty((M, M), np.float64) if with_image else None
        a, b = C.c_double(), C.c_double()
        self._ck(lib().mcao_get_psf(self.h, q, out.ctypes.data if with_image else None, M * M if with_image else 0,
                                    C.byref(a), C.byref(b)))
        return out, a.value, b.value

    def reset_psf(self):
        self._ck(lib().mcao_reset_psf(self.h))

    def get_state(self) -> bytes:
        n = self.query(Q_STATE)
        buf = (C.c_char * n)()
        self._ck(lib().mcao_get_state(self.h, buf, n))
        return bytes(buf)

    def set_state(self, blob: bytes):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        self._ck(lib().mcao_set_state(self.h, buf, len(blob)))

    def set_profiling(self, on: bool, stages=None):
        """Stage profiler on or off; with stages (names from STAGES), time only those."""
        if stages is None:
            self._ck(lib().mcao_set_profiling(self.h, int(on)))
        else:
            mask = sum(1 << STAGES.index(s) for s in stages) if on else 0
            self._ck(lib().mcao_set_profiling_stages(self.h, mask))

    def get_profile(self):
        ms = (C.c_double * len(STAGES))()
        cnt = (C.c_int64 * len(STAGES))()
        lps = C.c_int64()
        self._ck(lib().mcao_get_profile(self.h, ms, cnt, len(STAGES), C.byref(lps)))
        return ({s: ms[i] for i, s in enumerate(STAGES)}, {s: cnt[i] for i, s in enumerate(STAGES)}, lps.value)

    def get_timeline(self):
        """Launch timeline of the profiled steps (read before get_profile, which clears it):
        a list of (step, stage name, start ms, end ms), times relative to each step's first
        launch."""
        tot = C.c_size_t()
        self._ck(lib().mcao_get_timeline(self.h, None, None, None, None, 0, C.byref(tot)))
        n = tot.value
        stg = (C.c_int32 * max(n, 1))()
        t0 = (C.c_double * max(n, 1))()
        t1 = (C.c_double * max(n, 1))()
        stp = (C.c_int32 * max(n, 1))()
        self._ck(lib().mcao_get_timeline(self.h, stg, t0, t1, stp, n, C.byref(tot)))
        return [(stp[i], STAGES[stg[i]], t0[i], t1[i]) for i in range(n)]


def reconstruct_noalloc(R, s, c, gain: float, stream=None) -> None:
    """c <- c + gain R s with the allocation-free entry point.  R is a float32 CUDA tensor of n_cmd
    rows with unit column stride whose first s.numel() columns are used (its row stride is the
    leading dimension, so a column slice of a padded matrix works); s [n_slopes] and c [n_cmd] are
    contiguous float32 CUDA tensors, all on the current device.  Queued on ``stream`` (torch stream
    or raw handle; default: the current torch stream)."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("R", R), ("s", s), ("c", c)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
            raise McaoError(1, f"{name} must be a float32 CUDA tensor")
        if t.device.index != dev:
            raise McaoError(1, f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    if R.dim() != 2 or R.stride(1) != 1:
        raise McaoError(1, "R must be a 2-D tensor with unit column stride")
    if not (s.is_contiguous() and c.is_contiguous()):
        raise McaoError(1, "s and c must be contiguous")
    n_cmd, n_slopes, ld = R.shape[0], s.numel(), R.stride(0)
    if R.shape[1] < n_slopes or c.numel() != n_cmd:
        raise McaoError(2, f"R is {tuple(R.shape)}, s has {n_slopes} and c {c.numel()} elements")
    if stream is None:
        stream = torch.cuda.current_stream()
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    buf = C.create_string_buffer(256)
    st = lib().mcao_reconstruct_noalloc(R.data_ptr(), n_cmd, n_slopes, ld, s.data_ptr(), c.data_ptr(),
                                        float(gain), C.c_void_p(ptr), buf, 256)
    if st != 0:
        raise McaoError(st, buf.value.decode())


def tikhonov_reconstructor(D, alpha: float, fp64: bool = False, stream=None):
    """Control matrix R = -(D^T D + lambda I)^-1 D^T, lambda = alpha tr(D^T D) / n_cmd, computed in FP64
    on the GPU (mcao_tikhonov_reconstructor).  D: CUDA float32 tensor [n_slopes][n_cmd] with unit column
    stride (its row stride is the leading dimension).  Returns (R, lambda), R a CUDA tensor
    [n_cmd][n_slopes] of float32 (or float64 with fp64=True)."""
    import torch
    if not (isinstance(D, torch.Tensor) and D.is_cuda and D.dtype == torch.float32 and D.dim() == 2
            and D.stride(1) == 1):
        raise McaoError(1, "D must be a CUDA float32 tensor [n_slopes][n_cmd] with unit column stride")
    n_slopes, n_cmd = D.shape
    R = torch.empty((n_cmd, n_slopes), dtype=torch.float64 if fp64 else torch.float32, device=D.device)
    if stream is None:
        stream = torch.cuda.current_stream()
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    lam = C.c_double()
    buf = C.create_string_buffer(256)
    st = lib().mcao_tikhonov_reconstructor(D.data_ptr(), n_slopes, n_cmd, D.stride(0), float(alpha), R.data_ptr(),
                                           n_slopes, int(bool(fp64)), C.c_void_p(ptr), C.byref(lam), buf, 256)
    if st != 0:
        raise McaoError(st, buf.value.decode())
    return R, lam.value


def make_sim(cfg: dict, screens, R, s_ref=None, keep_frames: bool = False, stream=None,
             r_dtype: int = DTYPE_F32, n_real: int = 1) -> Sim:
    """Create a simulation and load the atmosphere, the DMs and the reconstructor (stored in the
    element format r_dtype).  With n_real > 1, screens is a list of n_real screen lists (one per
    realization)."""
    s = Sim(cfg, keep_frames=keep_frames, stream=stream, n_real=n_real)
    if n_real > 1:
        for r in range(n_real):
            s.load_atmosphere(screens[r], realization=r)
        s.set_realization(0)
    else:
        s.load_atmosphere(screens)
    s.load_dms()
    s.load_reconstructor(R, s_ref, dtype=r_dtype)
    return s


def step_group(sims, n: int = 1):
    """Advance simulations of any configurations together (mcao_step_group): one graph launch
    per step holding every simulation's step."""
    arr = (C.c_void_p * len(sims))(*[s.h for s in sims])
    st = lib().mcao_step_group(arr, len(sims), int(n))
    if st != 0:
        bad = next((s for s in sims if lib().mcao_last_error(s.h)), sims[0])
        raise McaoError(st, lib().mcao_last_error(bad.h).decode())


def _sensing_function():
    import torch

    class SensingFunction(torch.autograd.Function):
        """Noise-free slopes as a differentiable function of the DM commands: forward sets the
        commands and measures (mcao_measure), backward is the vector-Jacobian product at the
        same commands (mcao_slopes_vjp)."""

        @staticmethod
        def forward(ctx, commands, sim):
            c = commands.detach().to("cpu", torch.float32).numpy()
            sim.set_commands(c)
            s = sim.measure(noise=False)
            ctx.sim = sim
            ctx.c = c
            return torch.from_numpy(s.copy()).to(commands.device)

        @staticmethod
        def backward(ctx, g):
            ctx.sim.set_commands(ctx.c)
            gc, _ = ctx.sim.slopes_vjp(g)
            return gc.to(g.device), None

    return SensingFunction


_SENSING = None


def sensing(sim: "Sim", commands):
    """slopes = sensing(sim, commands): autograd-aware noise-free measurement at the current step
    (sets the simulation's commands; their controller memory restarts as after set_commands)."""
    global _SENSING
    if _SENSING is None:
        _SENSING = _sensing_function()
    return _SENSING.apply(commands, sim)


def generate_screen(n: int, pixel: float, r0: float, L0: float, seed: int, stream=None):
    """An n x n von Karman phase screen (rad) generated on the device by mcao_generate_screen;
    returns a CUDA float32 tensor."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    out = torch.empty((n, n), dtype=torch.float32, device="cuda")
    err = C.create_string_buffer(256)
    st = lib().mcao_generate_screen(int(n), float(pixel), float(r0), float(L0), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                    C.c_void_p(out.data_ptr()), C.c_void_p(ptr), err, 256)
    if st != 0:
        raise McaoError(st, err.value.decode())
    return out


def quantize_rows(R, dtype: int, stream=None):
    """(codes, scales) of a CUDA float32 matrix R [rows][cols] in a reduced format, computed on the
    device by mcao_quantize_rows: uint16 bfloat16 codes, or uint8 FP8 E4M3 codes with a float32
    scale per row (scales is None for bfloat16)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    rows, cols = R.shape
    codes = torch.empty((rows, cols), dtype=torch.int16 if dtype == DTYPE_BF16 else torch.uint8, device=R.device)
    scales = torch.empty(rows, dtype=torch.float32, device=R.device) if dtype == DTYPE_FP8_E4M3 else None
    err = C.create_string_buffer(256)
    st = lib().mcao_quantize_rows(C.c_void_p(R.data_ptr()), rows, cols, R.stride(0), int(dtype),
                                  C.c_void_p(codes.data_ptr()), C.c_void_p(scales.data_ptr() if scales is not None else 0),
                                  C.c_void_p(ptr), err, 256)
    if st != 0:
        raise McaoError(st, err.value.decode())
    return codes, scales
