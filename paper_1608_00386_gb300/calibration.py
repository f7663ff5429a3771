"""DM misregistration fit from an interaction matrix ("Conclusions": the rotation of the DM and its
modal basis with respect to the sensors; also translation and magnification).

The model interaction matrix D(p) of a DM moved by p = (shift_x, shift_y, rotation,
magnification) is the exact Jacobian computed on the device (mcao_set_misregistration, then
mcao_interaction_matrix).  The fit minimises ||D(p) - D_meas||_F^2 by damped Gauss-Newton
iterations; the sensitivities dD/dp_k are central differences of the model matrix.  The large
reductions run as torch operations on the device; the 4 x 4 normal equations are solved on the
host.
"""
from __future__ import annotations

import numpy as np


def fit_misregistration(sim, D_meas, dm: int, p0=(0.0, 0.0, 0.0, 1.0), steps=None, iters: int = 10,
                        tol: float = 1e-7, damping: float = 1e-6, cmd_cols=None):
    """Fit DM dm's misregistration so that sim's model interaction matrix matches D_meas (a CUDA
    tensor [n_slopes][n_commands], or only the columns cmd_cols; by default the columns of DM
    dm, the only ones its misregistration changes).  The simulation's other state
    (commands, step, the other DMs) sets the operating point.  Returns (p, history) with p the
    fitted (shift_x m, shift_y m, rotation rad, magnification) and history the relative residual
    per iteration; leaves the DM at p."""
    import torch
    pitch = float(sim.cfg["dms"][dm]["pitch"])
    h = np.asarray(steps if steps is not None else (0.01 * pitch, 0.01 * pitch, 1e-3, 1e-3), dtype=np.float64)
    dev = D_meas.device   # the device the model matrices live on
    if cmd_cols is None:
        # the DM's own block of the command vector: a contiguous column range (a view, no copy)
        n_valid = [int(np.count_nonzero(d["valid"])) for d in sim.cfg["dms"]]
        cols = slice(sum(n_valid[:dm]), sum(n_valid[:dm + 1]))
        n_cols = n_valid[dm]
    else:
        cols = torch.as_tensor(np.asarray(cmd_cols), device=dev, dtype=torch.long)
        n_cols = cols.numel()
    D_meas = D_meas.to(dtype=torch.float32)
    if D_meas.shape[1] != n_cols:
        D_meas = D_meas[:, cols]
    nrm = float(torch.linalg.vector_norm(D_meas))

    def model(p):
        sim.set_misregistration(dm, *[float(x) for x in p])
        return sim.interaction_matrix()[:, cols]

    p = np.asarray(p0, dtype=np.float64).copy()
    history = []
    for _ in range(iters):
        r = model(p) - D_meas
        history.append(float(torch.linalg.vector_norm(r)) / nrm)
        J = []
        for k in range(4):
            e = np.zeros(4)
            e[k] = h[k]
            J.append((model(p + e) - model(p - e)) / (2.0 * h[k]))
        A = np.zeros((4, 4))
        b = np.zeros(4)
        for k in range(4):
            b[k] = float(torch.sum(J[k].double() * r.double()))
            for l in range(k, 4):
                A[k, l] = A[l, k] = float(torch.sum(J[k].double() * J[l].double()))
        A += damping * np.diag(np.diag(A))
        delta = -np.linalg.solve(A, b)
        p += delta
        del J, r
        if np.all(np.abs(delta) <= tol * np.maximum(1.0, np.abs(p)) + np.array([1e-6 * pitch, 1e-6 * pitch, 1e-8, 1e-8])):
            break
    history.append(float(torch.linalg.vector_norm(model(p) - D_meas)) / nrm)   # leaves the DM at p
    return tuple(float(x) for x in p), history
