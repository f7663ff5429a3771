"""DM misregistration fit from an interaction matrix ("Conclusions": the rotation of the DM and its
modal basis with respect to the sensors; also translation and magnification).

The model interaction matrix D(p) of a DM moved by p = (shift_x, shift_y, rotation,
magnification) is the exact Jacobian of the noise-free slopes with respect to the DM's commands.
The fit minimises ||D(p) - D_meas||_F^2 by damped Gauss-Newton iterations.  Every iteration's
normal equations (the 4 x 4 matrix JtJ and the vector Jte, with the analytic derivatives dD/dp)
come from one library call, mcao_misreg_normal_equations, whose kernels form them without
building any model matrix; this module only solves the 4 x 4 system and updates p.
"""
from __future__ import annotations

import math

import numpy as np


def dm_columns(sim, D, dm: int):
    """The columns of DM dm's commands in an interaction matrix D [n_slopes][n_commands] (a view)."""
    n_valid = [int(np.count_nonzero(d["valid"])) for d in sim.cfg["dms"]]
    c0 = sum(n_valid[:dm])
    return D[:, c0:c0 + n_valid[dm]]


def fit_misregistration(sim, D_meas, dm: int, p0=(0.0, 0.0, 0.0, 1.0), iters: int = 10, tol: float = 1e-7,
                        damping: float = 1e-6):
    """Fit DM dm's misregistration so that sim's model interaction matrix matches D_meas, a CUDA
    float32 tensor [n_slopes][n_commands] (the full matrix) or [n_slopes][the DM's commands].  The
    simulation's other state (commands, step, the other DMs) sets the operating point.  Returns
    (p, history) with p the fitted (shift_x m, shift_y m, rotation rad, magnification) and history
    the relative residual ||D(p) - D_meas|| / ||D_meas|| per iteration; leaves the DM at p."""
    pitch = float(sim.cfg["dms"][dm]["pitch"])
    n_dm = int(np.count_nonzero(sim.cfg["dms"][dm]["valid"]))
    if D_meas.shape[1] != n_dm:
        D_meas = dm_columns(sim, D_meas, dm)
    p = np.asarray(p0, dtype=np.float64).copy()
    history = []
    floor = np.array([1e-6 * pitch, 1e-6 * pitch, 1e-8, 1e-8])
    for _ in range(iters):
        sim.set_misregistration(dm, *[float(x) for x in p])
        JtJ, Jte, cost, msq = sim.misreg_normal_equations(dm, D_meas)
        history.append(math.sqrt(cost / msq))
        delta = -np.linalg.solve(JtJ + damping * np.diag(np.diag(JtJ)), Jte)
        p += delta
        if np.all(np.abs(delta) <= tol * np.maximum(1.0, np.abs(p)) + floor):
            break
    sim.set_misregistration(dm, *[float(x) for x in p])
    _, _, cost, msq = sim.misreg_normal_equations(dm, D_meas)
    history.append(math.sqrt(cost / msq))
    return tuple(float(x) for x in p), history
