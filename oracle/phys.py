"""FP64 oracle of the physics-informed wind loss (Sec. 3.4) and of the pieces
of the wind inversion loop around it.

TEST INFRASTRUCTURE ONLY: the CUDA path is checked against these functions;
only tests/, the smoke check in __graft_entry__.py and bench.py's reference
leg may import this module. Nothing here is shared with the CUDA library.

What it computes, in numpy float64:
  - lbm_sample_velocity / sample_velocity_field: the LBM macroscopic velocity
    (Eq. lbm_sum_v2, via the lattice oracle's moments, or any cell field such
    as the HOME-LBM oracle's) trilinearly interpolated at arbitrary points of
    the unit cube. Reading: lattice cell c spans [c/n, (c+1)/n)
    (the cell of Eq. point2voxel with dx = 1/n), its velocity sits at the
    cell centre (c + 1/2)/n; solid cells have u = 0; points are clamped to
    the box of cell centres.
  - phys_loss: Sec. 3.4's L_phys = |D_recon - (D_recon . D_guide) D_guide|^2
    summed over the wind-grid nodes of one keyframe. Reading: D_recon is the
    node's wind force, D_guide the unit direction of the LBM velocity there;
    nodes where the flow is (almost) still, |u| <= eps, give no guidance and
    add nothing. With P = I - d d^T (a projector for unit d) the term is
    |P F|^2 and its gradient is 2 P F.
  - drag_force: Sec. 3.4's drag relation F_w = 1/2 rho_w C_D |v|^2 v/|v|,
    with all constants folded into one scale: F = scale |u| u.
  - position_loss: the trajectory term weight * sum_p |x_p - x_p*|^2 and its
    gradient 2 weight (x - x*).
  - adam_step: Adam (Kingma and Ba, 2015) with bias correction.
  - vector_adam_step: VectorAdam (Ling, Sharp and Jacobson, 2022): Adam whose
    second moment is taken on the squared norm of each 3-vector's gradient.
  - cos_sim, nmse: the scores of the wind-force-field evaluation (App. E.2,
    the CosSim / NMSE table): both on force vectors normalised to unit length.
"""
import numpy as np

from . import lbm_macroscopic


def lbm_sample_velocity(shape, f, pos, solid=None, force=(0.0, 0.0, 0.0)):
    """u[3][m] at positions pos[3][m] of the unit cube, from populations f
    (natural order, f[q][cell] unshifted, as the lattice oracle stores them)."""
    _, u = lbm_macroscopic(shape, f, force, solid)
    return sample_velocity_field(shape, u, pos)


def sample_velocity_field(shape, u, pos):
    """u[3][m] at positions pos[3][m] of a cell-centred velocity field u
    [3][nz*ny*nx] (solid cells already at rest), trilinear between cell
    centres, clamped to their box."""
    nx, ny, nz = shape
    u = np.asarray(u, np.float64).reshape(3, nz, ny, nx)
    pos = np.asarray(pos, np.float64)
    m = pos.shape[1]
    out = np.zeros((3, m))
    dims = (nx, ny, nz)
    for p in range(m):
        i0, t = [0, 0, 0], [0.0, 0.0, 0.0]
        for a in range(3):
            n = dims[a]
            s = min(max(pos[a, p] * n - 0.5, 0.0), n - 1.0)
            i = min(int(np.floor(s)), n - 2)
            i0[a], t[a] = i, s - i
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    w = ((t[0] if cx else 1 - t[0]) * (t[1] if cy else 1 - t[1]) *
                         (t[2] if cz else 1 - t[2]))
                    out[:, p] += w * u[:, i0[2] + cz, i0[1] + cy, i0[0] + cx]
    return out


def phys_loss(values, guide_u, eps=1e-6):
    """(L_phys, dL/dvalues) of one keyframe: values [m][3] wind forces at the
    nodes, guide_u [3][m] LBM velocities there."""
    F = np.asarray(values, np.float64).reshape(-1, 3)
    u = np.asarray(guide_u, np.float64).reshape(3, -1).T
    loss = 0.0
    g = np.zeros_like(F)
    for k in range(F.shape[0]):
        norm = np.sqrt(u[k] @ u[k])
        if norm <= eps:
            continue
        d = u[k] / norm
        r = F[k] - (F[k] @ d) * d
        loss += r @ r
        g[k] = 2.0 * r
    return loss, g


def drag_force(u, scale):
    """values [m][3] = scale |u| u for velocities u [3][m]."""
    u = np.asarray(u, np.float64).reshape(3, -1).T
    speed = np.sqrt(np.sum(u * u, axis=1))
    return scale * speed[:, None] * u


def position_loss(x, x_target, weight=1.0):
    """(weight * sum |x - x*|^2, its gradient [3][n]) for x, x* [3][n]."""
    d = np.asarray(x, np.float64) - np.asarray(x_target, np.float64)
    return weight * float(np.sum(d * d)), 2.0 * weight * d


def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step >= 1); returns (param, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def vector_adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One VectorAdam update of param [n][3] (m [n][3], v [n]); returns
    (param, m, v)."""
    grad = np.asarray(grad, np.float64).reshape(-1, 3)
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * np.sum(grad * grad, axis=1)
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh)[:, None] + eps), m, v


def _unit_pairs(rec, gt, eps):
    """Unit vectors of the locations where both fields have a direction."""
    a = np.asarray(rec, np.float64).reshape(-1, 3)
    b = np.asarray(gt, np.float64).reshape(-1, 3)
    na, nb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
    keep = (na > eps) & (nb > eps)
    return a[keep] / na[keep, None], b[keep] / nb[keep, None]


def cos_sim(rec, gt, eps=1e-12):
    """The evaluation's CosSim: the mean over grid locations (and time steps)
    of F_gt^ . F_rec^, each force normalised to unit length. Reading: a
    location where either force is zero has no direction and is left out."""
    a, b = _unit_pairs(rec, gt, eps)
    return float(np.mean(np.sum(a * b, axis=1)))


def nmse(rec, gt, eps=1e-12):
    """The evaluation's NMSE: the mean of |F_gt^ - F_rec^|^2 over the same
    normalised vectors (range [0, 4]; for unit vectors it equals
    2 - 2 CosSim)."""
    a, b = _unit_pairs(rec, gt, eps)
    return float(np.mean(np.sum((a - b) ** 2, axis=1)))
