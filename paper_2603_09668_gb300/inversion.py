"""The physics-informed wind inversion loop (Sec. 3.3 and 3.4) and the
LBM-driven forward simulation it is scored against, run on the library's
kernels; this module only orders the calls and owns the buffers.

Forward simulation (Sec. 3.4, wind field evolution): per frame interval the
particles are voxelized into the lattice's solid mask (Eq. point2voxel), the
lattice advances, its velocity is sampled at the wind-grid nodes, the drag
relation turns it into a wind acceleration (wind_drag_force), and the MPM
runs the interval's substeps under that force, held constant over the
interval (one keyframe).

Inversion (Sec. 3.3): the intervals are solved one after another. For each,
the force keyframe starts at zero and Adam minimises

    w_data * sum_p |x_p(end) - x_p_observed|^2  +  lambda * L_phys,

the first gradient coming from the checkpointed MPM adjoint
(mpm_segment_adjoint, one call per checkpoint segment) and the second from
wind_phys_loss against the lattice velocity of that interval (the guide, from
a lattice whose inlet points along the assumed wind-source direction). The
optimised force then advances the state, which starts the next interval.
The update is VectorAdam by default: per-component Adam moves every
component of every node by about the learning rate whatever its gradient's
size, which scrambles the per-node directions the evaluation scores; plain
Adam stays available (optimizer="adam").
The data term is either the squared distance to observed particle positions
or, with a Gaussian renderer and cameras (RenderObservation), L_render's L1
term between the particle-bound Gaussians drawn from the simulated state
and the observed images, its gradient taken through the renderer
(gs_render_backward) into the MPM adjoint's dL/dx and dL/dF.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import binding as B
from .inputs import rest_state, wind_node_positions


class LbmGuide:
    """A lattice over the unit cube (nx = ny = nz, so one voxel size dx = 1/nx
    serves Eq. point2voxel and the velocity sampler) with an inlet at x = 0,
    evolved alongside the object, and its velocity at the nf^3 wind nodes.
    model "home" runs HOME-LBM (the paper's wind solver, Sec. 3.4), "bgk" the
    BGK step."""

    def __init__(self, n_cells: int, tau: float, u_inlet, nf: int, device="cuda",
                 model: str = "home"):
        if model not in ("home", "bgk"):
            raise ValueError(f"unknown lattice model {model!r}")
        self.shape = (n_cells, n_cells, n_cells)
        self.n_cells = n_cells
        self.u_inlet = tuple(float(c) for c in u_inlet)
        self.nf = nf
        self.model = model
        self.lbm = B.LBM(self.shape, tau, u_inlet=self.u_inlet, bc_x=1)
        if model == "home":
            self.f = self.lbm.moments(device)
            self.lbm.home_init(self.f, 1.0, self.u_inlet)
        else:
            self.f = self.lbm.lattice(device)
            self.lbm.init_equilibrium(self.f, 1.0, self.u_inlet)
        self.solid = torch.zeros((n_cells, n_cells, n_cells), dtype=torch.uint8, device=device)
        self.nodes = torch.from_numpy(wind_node_positions(nf)).to(device)
        self.u = torch.empty((3, nf ** 3), dtype=torch.float32, device=device)

    def advance(self, x: torch.Tensor, steps: int) -> torch.Tensor:
        """Voxelize the particles x [3][n], run `steps` lattice steps and return
        the velocity at the wind nodes [3][nf^3] (a view of the guide's buffer,
        overwritten by the next call)."""
        B.voxelize_particles(x, self.shape, 1.0 / self.n_cells, self.solid)
        if self.model == "home":
            if steps > 0:
                self.lbm.home_step(self.f, self.solid, steps)
            self.lbm.home_sample_velocity(self.f, self.solid, self.nodes, self.u)
        else:
            if steps > 0:
                self.lbm.step(self.f, self.solid, steps)
            self.lbm.sample_velocity(self.f, self.solid, self.nodes, self.u)
        return self.u

    def close(self):
        self.lbm.close()


def _wind(values: torch.Tensor) -> B.WindField:
    # one keyframe: the force is constant over the interval
    return B.WindField(values, 1.0)


def simulate_wind_driven(mpm: B.MPM, guide: LbmGuide, state: B.MpmState, pinned, n_intervals: int,
                         substeps: int, lbm_steps: int, drag_scale: float, t0: float = 0.0):
    """Advance `state` in place through n_intervals intervals of `substeps`
    substeps, each driven by the drag force of the guide lattice's velocity.
    Returns (forces [n_intervals][nf^3][3], positions [n_intervals][3][n] at
    the end of each interval)."""
    nf = guide.nf
    forces = torch.empty((n_intervals, nf ** 3, 3), dtype=torch.float32, device=state.x.device)
    xs = torch.empty((n_intervals,) + tuple(state.x.shape), dtype=torch.float32,
                     device=state.x.device)
    t = t0
    for k in range(n_intervals):
        u = guide.advance(state.x, lbm_steps)
        B.wind_drag_force(u, drag_scale, forces[k])
        mpm.rollout(state, pinned, None, _wind(forces[k].view(1, nf, nf, nf, 3)), t, substeps, 0)
        xs[k].copy_(state.x)
        t += substeps * mpm.dt
    return forces, xs


@dataclass
class RenderObservation:
    """Views of the particle-bound Gaussians: one renderer, its cameras, the
    Gaussians' rest covariances [6][n], colours [3][n] and opacities [n].
    The image term is L_render's per view, (1 - lambda_ssim) L1 + lambda_ssim
    D-SSIM with lambda_ssim = 0.1 (Sec. 3.3)."""
    renderer: B.GaussianRenderer
    cameras: list
    sigma0: torch.Tensor
    color: torch.Tensor
    opacity: torch.Tensor
    lambda_ssim: float = 0.1

    def images(self, state: B.MpmState) -> torch.Tensor:
        """[n_views][3][H][W] images of the state."""
        r = self.renderer
        out = torch.empty((len(self.cameras), 3, r.height, r.width), dtype=torch.float32,
                          device=state.x.device)
        for v, cam in enumerate(self.cameras):
            r.render(cam, state.x, state.F, self.sigma0, self.color, self.opacity, out[v])
        return out

    def loss(self, state: B.MpmState, target: torch.Tensor, weight: float, loss: torch.Tensor,
             g: B.MpmState, scratch: torch.Tensor, workspace: torch.Tensor):
        """loss += weight 3 H W times L_render summed over the views (with
        weight = 1 / (3 H W): (1 - lambda) mean |image - target| + lambda
        D-SSIM per view); g.x and g.F += its gradient (each view drawn, then
        differentiated right away)."""
        r = self.renderer
        lam = self.lambda_ssim
        npix = 3 * r.height * r.width
        for v, cam in enumerate(self.cameras):
            r.render(cam, state.x, state.F, self.sigma0, self.color, self.opacity, scratch[0])
            scratch[1].zero_()
            B.image_l1_loss(scratch[0], target[v], loss, (1.0 - lam) * weight, scratch[1])
            if lam > 0.0:
                B.image_dssim_loss(scratch[0], target[v], loss, lam * weight * npix, scratch[1],
                                   workspace)
            r.backward(cam, state.x, state.F, self.sigma0, self.color, self.opacity, scratch[1],
                       g.x, g.F)


@dataclass
class InversionResult:
    values: torch.Tensor   # [n_intervals][nf^3][3] reconstructed force per interval
    history: torch.Tensor  # [n_intervals][iters][2]: (data term, lambda * L_phys) per iteration
    x_end: torch.Tensor    # [n_intervals][3][n] positions after each committed interval
    guides: torch.Tensor   # [n_intervals][3][nf^3] lattice velocity used as the guide


class WindInversion:
    """Sequential per-interval reconstruction of the wind force field.

    iters Adam iterations per interval (learning rate lr), each one forward
    pass of `substeps` substeps with a checkpoint every `every` substeps and
    one reverse pass. w_data weights the position term (default 1 / (n h^2)
    with h the grid spacing: the mean squared position error in grid cells);
    lam_phys weights L_phys; optimizer is "vector_adam" or "adam"."""

    def __init__(self, mpm: B.MPM, guide: LbmGuide, substeps: int, every: int, iters: int,
                 lr: float, lam_phys: float, w_data: Optional[float] = None, eps_guide=1e-6,
                 optimizer: str = "vector_adam"):
        if substeps < 1 or every < 1 or iters < 1:
            raise ValueError("substeps, every and iters must be >= 1")
        if optimizer not in ("vector_adam", "adam"):
            raise ValueError(f"unknown optimizer {optimizer!r}")
        self.optimizer = optimizer
        self.mpm, self.guide = mpm, guide
        self.substeps, self.every, self.iters = substeps, every, iters
        self.lr, self.lam_phys, self.w_data, self.eps_guide = lr, lam_phys, w_data, eps_guide

    def reconstruct(self, state0: B.MpmState, pinned, x_observed: torch.Tensor,
                    lbm_steps: int, t0: float = 0.0,
                    views: Optional[RenderObservation] = None) -> InversionResult:
        """x_observed: the observation at the end of each interval, positions
        [n_intervals][3][n], or with views the images [n_intervals][n_views][3]
        [H][W] (then w_data defaults to 1 / (3 H W), the mean L1 per view).
        state0 is not modified."""
        mpm, guide, nf = self.mpm, self.guide, self.guide.nf
        dev = state0.x.device
        n, K, S, every = state0.n, x_observed.shape[0], self.substeps, self.every
        if views is None:
            w_data = self.w_data if self.w_data is not None else mpm.n_grid ** 2 / max(n, 1)
        else:
            r = views.renderer
            w_data = self.w_data if self.w_data is not None else 1.0 / (3 * r.width * r.height)
            scratch = torch.empty((2, 3, r.height, r.width), dtype=torch.float32, device=dev)
            ssim_ws = torch.empty(10 * 3 * r.height * r.width, dtype=torch.float32, device=dev)
        segs = [(k0, min(S, k0 + every)) for k0 in range(0, S, every)]

        values = torch.zeros((K, nf ** 3, 3), dtype=torch.float32, device=dev)
        history = torch.zeros((K, self.iters, 2), dtype=torch.float32, device=dev)
        x_end = torch.empty((K, 3, n), dtype=torch.float32, device=dev)
        guides = torch.empty((K, 3, nf ** 3), dtype=torch.float32, device=dev)
        g_values = torch.empty((nf ** 3, 3), dtype=torch.float32, device=dev)
        m_buf = torch.empty_like(g_values)
        vec = self.optimizer == "vector_adam"
        v_buf = torch.empty(nf ** 3 if vec else (nf ** 3, 3), dtype=torch.float32, device=dev)
        state = state0.clone()
        run = B.MpmState.empty_like(state0)
        ckpts = [B.MpmState.empty_like(state0) for _ in segs]
        g = B.MpmState.empty_like(state0)
        tape = torch.empty(max(every - 1, 1) * 24 * max(n, 1), dtype=torch.float32, device=dev)

        t = t0
        for k in range(K):
            guides[k].copy_(guide.advance(state.x, lbm_steps))
            val = values[k]
            wind = _wind(val.view(1, nf, nf, nf, 3))
            m_buf.zero_()
            v_buf.zero_()
            for it in range(self.iters):
                # forward with a checkpoint at the start of every segment
                for c, a in zip(run, state):
                    c.copy_(a)
                for (k0, k1), ck in zip(segs, ckpts):
                    for c, a in zip(ck, run):
                        c.copy_(a)
                    mpm.rollout(run, pinned, None, wind, t + k0 * mpm.dt, k1 - k0, 0)
                # losses and the reverse pass
                for a in g:
                    a.zero_()
                g_values.zero_()
                if views is None:
                    B.position_loss(run.x, x_observed[k], history[k, it, 0:1], w_data, g.x)
                else:
                    views.loss(run, x_observed[k], w_data, history[k, it, 0:1], g, scratch,
                               ssim_ws)
                for (k0, k1), ck in zip(reversed(segs), reversed(ckpts)):
                    mpm.segment_adjoint(ck, tape, g, pinned, wind, t + k0 * mpm.dt, k1 - k0,
                                        g_values.view(1, nf, nf, nf, 3))
                if self.lam_phys > 0.0:
                    B.wind_phys_loss(val, guides[k], history[k, it, 1:2], g_values,
                                     self.eps_guide, self.lam_phys)
                if vec:
                    B.vector_adam_step(val, g_values, m_buf, v_buf, it + 1, self.lr)
                else:
                    B.adam_step(val, g_values, m_buf, v_buf, it + 1, self.lr)
            # commit the interval with the optimised force
            mpm.rollout(state, pinned, None, wind, t, S, 0)
            x_end[k].copy_(state.x)
            t += S * mpm.dt
        return InversionResult(values, history, x_end, guides)


def field_scores(rec: torch.Tensor, gt: torch.Tensor, eps: float = 1e-12):
    """(CosSim, NMSE) of rec against gt over all intervals and nodes where both
    forces have a direction (App. E.2), from wind_field_scores."""
    sums = B.wind_field_scores(rec.contiguous(), gt.contiguous(), eps=eps)
    s = sums.cpu().numpy().astype(np.float64)
    if s[2] == 0:
        return float("nan"), float("nan")
    return float(s[0] / s[2]), float(s[1] / s[2])


def rotate_about_y(vec, degrees):
    """vec rotated by `degrees` about the y axis (an assumed wind-source
    direction that is off by that angle)."""
    a = np.deg2rad(degrees)
    x, y, z = vec
    return (float(np.cos(a) * x + np.sin(a) * z), float(y), float(-np.sin(a) * x + np.cos(a) * z))


@dataclass
class SyntheticCase:
    mpm: B.MPM
    state0: B.MpmState
    pinned: Optional[torch.Tensor]
    gt_forces: torch.Tensor  # [n_intervals][nf^3][3]
    x_obs: torch.Tensor      # [n_intervals][3][n]
    guide: LbmGuide          # the inversion's guide lattice (assumed inlet)

    def close(self):
        self.guide.close()
        self.mpm.close()


def prepare_synthetic(case: dict, device="cuda") -> SyntheticCase:
    """Ground truth of a synthetic case (inputs.inversion_case): the forward
    simulation with the true inlet from the sheet at rest, and a fresh guide
    lattice for the inversion whose inlet is rotated by the case's error."""
    sc = case["scene"]
    nf, K, S = case["nf"], case["n_intervals"], case["substeps"]
    state0 = B.MpmState(*(torch.from_numpy(np.asarray(a, np.float32)).to(device)
                          for a in rest_state(sc.x)))
    pinned = torch.from_numpy(sc.pinned).to(device) if sc.pinned is not None else None
    mpm = B.MPM.from_params(sc.params(), max_particles=sc.n)
    model = case.get("lbm_model", "home")
    gt_guide = LbmGuide(case["n_cells"], case["tau"], case["u_inlet"], nf, device, model)
    gt_forces, x_obs = simulate_wind_driven(mpm, gt_guide, state0.clone(), pinned, K, S,
                                            case["lbm_steps"], case["drag_scale"])
    gt_guide.close()
    guide = LbmGuide(case["n_cells"], case["tau"],
                     rotate_about_y(case["u_inlet"], case["inlet_error_deg"]), nf, device, model)
    return SyntheticCase(mpm, state0, pinned, gt_forces, x_obs, guide)


def sheet_views(case: dict, state0: B.MpmState, width: int = 128, height: int = 128):
    """Two views of the case's sheet (front, and 0.6 rad about y) with
    particle-bound Gaussians of the lattice spacing's size and a checkerboard
    of colours over the rest positions (texture makes motion visible)."""
    from .inputs import sheet_texture

    sc = case["scene"]
    dev = state0.x.device
    h = 0.6 / (case["nu"] - 1)  # the sheet's lattice spacing
    sigma0 = torch.zeros((6, sc.n), dtype=torch.float32, device=dev)
    sigma0[:3] = h * h
    color = torch.from_numpy(sheet_texture(sc.x)).to(dev)
    opacity = torch.full((sc.n,), 0.9, dtype=torch.float32, device=dev)
    centre = np.array([0.5, 0.6, 0.5])
    f = 1.25 * width
    cams = []
    for ang in (0.0, 0.6):
        R = np.array([[np.cos(ang), 0.0, np.sin(ang)], [0.0, 1.0, 0.0],
                      [-np.sin(ang), 0.0, np.cos(ang)]])
        T = np.array([0.0, 0.0, 1.5]) - R @ centre
        cams.append(B.camera(R, T, f, f, width / 2, height / 2, width, height))
    r = B.GaussianRenderer(sc.n, width, height)
    return RenderObservation(r, cams, sigma0, color, opacity)


def run_synthetic(case: dict, iters: int = 40, lr: float = 1.0, lam_phys: float = 0.1,
                  device="cuda", optimizer="vector_adam", observe: str = "positions",
                  w_data: Optional[float] = None):
    """prepare_synthetic, then the inversion from the same initial state,
    observing the particle positions or (observe="render") two rendered
    views of the ground-truth states. Returns a dict with the ground truth,
    the InversionResult and the scores."""
    syn = prepare_synthetic(case, device)
    inv = WindInversion(syn.mpm, syn.guide, case["substeps"], case["every"], iters, lr, lam_phys,
                        w_data=w_data, optimizer=optimizer)
    if observe == "render":
        views = sheet_views(case, syn.state0)
        K = syn.x_obs.shape[0]
        obs = torch.empty((K, len(views.cameras), 3, views.renderer.height, views.renderer.width),
                          dtype=torch.float32, device=syn.state0.x.device)
        # the observed images: the ground-truth states at the interval ends (F from a re-run)
        st = syn.state0.clone()
        nf = syn.guide.nf
        t = 0.0
        for k in range(K):
            wind = _wind(syn.gt_forces[k].view(1, nf, nf, nf, 3))
            syn.mpm.rollout(st, syn.pinned, None, wind, t, case["substeps"], 0)
            t += case["substeps"] * syn.mpm.dt
            obs[k] = views.images(st)
        res = inv.reconstruct(syn.state0, syn.pinned, obs, case["lbm_steps"], views=views)
        views.renderer.close()
    elif observe == "positions":
        res = inv.reconstruct(syn.state0, syn.pinned, syn.x_obs, case["lbm_steps"])
    else:
        raise ValueError(f"unknown observation {observe!r}")
    cos, nmse = field_scores(res.values, syn.gt_forces)
    out = dict(gt_forces=syn.gt_forces, x_obs=syn.x_obs, result=res, cos_sim=cos, nmse=nmse)
    syn.close()
    return out
