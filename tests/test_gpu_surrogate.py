"""GPU parity of the surrogate network (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 oracle, through the C-ABI.

The oracle receives the same BF16-rounded weights and features (as float64),
so the differences come from the BF16 storage of the hidden activations and
gradients: unit roundoff 2^-8 per stored value, a few roundings per layer,
giving about 1% relative L2 at the output. Tolerances: forward 2e-2, weight
gradients 5e-2 relative L2 per layer, features 1e-2 (one BF16 rounding),
re-equilibrated populations 1e-6 absolute (FP32 arithmetic on exact inputs)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def random_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(oracle.surr_num_params(), np.float32)
    for ws, bs, cin, cout in oracle.surr_layer_slices():
        p[ws] = rng.standard_normal(ws.stop - ws.start) * scale * np.sqrt(2.0 / (27 * cin))
        p[bs] = rng.standard_normal(cout) * 0.1
    return p


def oracle_params(p):
    """BF16-rounded weights, FP32 biases: what the GPU computes with."""
    q = np.asarray(p, np.float64).copy()
    for ws, bs, cin, cout in oracle.surr_layer_slices():
        q[ws] = bf16_round(p[ws])
    return q


def random_features(n, seed=1):
    rng = np.random.default_rng(seed)
    f = np.zeros((n ** 3, 16), np.float32)
    f[:, :5] = rng.standard_normal((n ** 3, 5)).astype(np.float32)
    return f


@pytest.mark.parametrize("n", [16, 32])
def test_forward_matches_oracle(n):
    p = random_params(seed=n)
    feats = random_features(n, seed=n + 1)
    s = B.Surrogate(n)
    s.set_params(to_dev(p))
    s.set_features(to_dev(feats))
    out = torch.empty((n ** 3, 16), device="cuda")
    s.forward(out)
    ref = oracle.surr_forward(n, oracle_params(p), bf16_round(feats))
    assert rel_l2(out.cpu().numpy()[:, :3].astype(np.float64), ref[:, :3]) <= 2e-2
    assert rel_l2(out.cpu().numpy().astype(np.float64), ref) <= 2e-2
    # the inference pass (all layers in one cooperative launch, grid barriers
    # between them; at n = 16 most CTAs own no tile and only pass the
    # barriers) computes the same tiles with the same arithmetic
    inf = torch.empty_like(out)
    for _ in range(2):
        s.forward(inf, keep_activations=False)
    s.device_status()
    a, b = inf.cpu().numpy(), out.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), np.abs(a - b).max()
    s.close()


def test_inference_pass_matches_the_layer_kernels_at_64():
    """At the 128^3 lattice's coarse size (64^3: every CTA owns 13-14 output
    slices, some across two tiles) the one-launch inference pass equals the
    per-layer kernels: the same tiles, the same arithmetic."""
    n = 64
    p = random_params(seed=11)
    feats = random_features(n, seed=12)
    s = B.Surrogate(n)
    s.set_params(to_dev(p))
    s.set_features(to_dev(feats))
    out = torch.empty((n ** 3, 16), device="cuda")
    s.forward(out)
    inf = torch.empty_like(out)
    for _ in range(3):
        s.forward(inf, keep_activations=False)
    s.device_status()
    a, b = inf.cpu().numpy(), out.cpu().numpy()
    assert np.isfinite(a).all() and np.abs(b).max() > 0
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), np.abs(a - b).max()
    s.close()


def test_backward_matches_oracle():
    n = 16
    p = random_params(seed=3)
    feats = random_features(n, seed=4)
    g_out = np.zeros((n ** 3, 16), np.float32)
    g_out[:, :3] = np.random.default_rng(5).standard_normal((n ** 3, 3)).astype(np.float32)
    s = B.Surrogate(n)
    s.set_params(to_dev(p))
    s.set_features(to_dev(feats))
    s.zero_grads()
    s.forward()
    s.set_output_grad(to_dev(g_out))
    s.backward()
    g = s.grads().cpu().numpy().astype(np.float64)
    ref = oracle.surr_backward(n, oracle_params(p), bf16_round(feats), bf16_round(g_out))
    for l, (ws, bs, cin, cout) in enumerate(oracle.surr_layer_slices()):
        assert rel_l2(g[ws], ref[ws]) <= 5e-2, (l, "W", rel_l2(g[ws], ref[ws]))
        assert rel_l2(g[bs], ref[bs]) <= 5e-2, (l, "b", rel_l2(g[bs], ref[bs]))
    s.close()


@pytest.mark.parametrize("u_ref", [(0.0, 0.0, 0.0), (0.045, 0.012, -0.018)])
def test_features_and_apply_match_oracle(u_ref):
    n = 16
    N = 2 * n
    shape = (N, N, N)
    c, w, _ = oracle.velocity_set()
    solid = inputs.random_mask(shape, 0.1, seed=6)
    rng = np.random.default_rng(7)
    u0 = np.array([0.05, 0.01, -0.02])
    feq = oracle.lbm_equilibrium(1.0, u0)
    f_plain = feq[:, None] + rng.uniform(-2e-3, 2e-3, (19, N ** 3))
    f_dev = to_dev((f_plain - w[:, None]).astype(np.float32).reshape(19, N, N, N))
    s = B.Surrogate(n)
    s.set_inlet(u_ref)
    s.features(f_dev, to_dev(solid).reshape(N, N, N))
    got = s.get_features().float().cpu().numpy().astype(np.float64)
    ref, rho, u = oracle.surr_features(n, f_plain.astype(np.float32).astype(np.float64), solid,
                                       u_ref)
    assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max()
    assert np.array_equal(got[:, 4], ref[:, 4])  # solid fractions are exact in BF16
    du = np.zeros((n ** 3, 16), np.float32)
    du[:, :3] = rng.standard_normal((n ** 3, 3)).astype(np.float32) * 1e-3
    f_out = f_dev.clone()
    s.apply(to_dev(solid).reshape(N, N, N), f_out, to_dev(du))
    f_ref = oracle.surr_apply(n, du, rho, u, f_plain, solid)
    got_f = f_out.reshape(19, -1).cpu().numpy().astype(np.float64) + w[:, None]
    fl = solid == 0
    assert np.abs(got_f[:, fl] - f_ref[:, fl]).max() <= 1e-6
    s.close()


def test_velocity_error_reduction():
    N = 24
    c, w, _ = oracle.velocity_set()
    rng = np.random.default_rng(8)
    fa = rng.uniform(-1e-3, 1e-3, (19, N ** 3)).astype(np.float32)
    fb = rng.uniform(-1e-3, 1e-3, (19, N ** 3)).astype(np.float32)
    solid = inputs.random_mask((N, N, N), 0.2, seed=9)
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    B.lbm_velocity_error(to_dev(fa), to_dev(fb), to_dev(solid), sums)
    _, ua = oracle.lbm_macroscopic((N, N, N), fa.astype(np.float64) + w[:, None], solid=solid)
    _, ub = oracle.lbm_macroscopic((N, N, N), fb.astype(np.float64) + w[:, None], solid=solid)
    e = np.sum((ua - ub) ** 2)
    r = np.sum(ub ** 2)
    assert sums[0].item() == pytest.approx(e, rel=1e-4)
    assert sums[1].item() == pytest.approx(r, rel=1e-4)


def test_training_fits_a_teacher_network():
    """Adam on the library's forward/backward kernels fits the outputs of a
    random teacher network of the same architecture."""
    n = 16
    feats = random_features(n, seed=10)
    teacher = random_params(seed=11, scale=0.5)
    target = oracle.surr_forward(n, oracle_params(teacher), bf16_round(feats)).astype(np.float32)
    s = B.Surrogate(n)
    s.set_params(to_dev(random_params(seed=12, scale=0.5)))
    s.set_features(to_dev(feats))
    tgt = to_dev(target)
    losses = []
    loss = torch.zeros(1, device="cuda")
    for step in range(1, 201):
        loss.zero_()
        s.forward()
        s.loss(tgt, loss)
        s.backward()
        s.adam(3e-3, step)
        if step in (1, 200):
            losses.append(loss.item())
    assert losses[1] < 0.1 * losses[0], losses
    s.close()


def test_chained_advance_matches_apply_and_features():
    """surr_advance_fine (u += out_scale * upsampled output, then the coarse
    features of the new state) against surr_apply (which re-equilibrates the
    lattice from the same upsampled update) and surr_features_fine."""
    n = 16
    N = 2 * n
    c, w, _ = oracle.velocity_set()
    solid = inputs.random_mask((N, N, N), 0.1, seed=13)
    rng = np.random.default_rng(14)
    feq = oracle.lbm_equilibrium(1.0, np.array([0.04, -0.01, 0.02]))
    f_plain = feq[:, None] + rng.uniform(-2e-3, 2e-3, (19, N ** 3))
    f_dev = to_dev((f_plain - w[:, None]).astype(np.float32).reshape(19, N, N, N))
    sol = to_dev(solid).reshape(N, N, N)
    s = B.Surrogate(n)
    s.set_params(to_dev(random_params(seed=15, scale=0.3)))
    s.features(f_dev, sol, 20.0)
    s.forward(keep_activations=False)  # the output the update upsamples
    f_apply = f_dev.clone()
    s.apply(sol, f_apply, None, 1e-3)
    s.advance_fine(1e-3, sol, 20.0)
    feats_adv = s.get_features().clone()
    f_adv = f_dev.clone()
    s.write_lattice(sol, f_adv)
    fl = torch.from_numpy(solid == 0).to("cuda").reshape(-1)
    d = (f_apply.reshape(19, -1)[:, fl] - f_adv.reshape(19, -1)[:, fl]).abs().max().item()
    assert d <= 1e-7, d
    s.features_fine(sol, 20.0)
    assert torch.equal(s.get_features(), feats_adv)
    s.device_status()
    s.close()


def test_chained_correction_adds_the_plain_defect():
    """surr_set_correction: with a network that predicts no change (zero
    parameters), one chained block after setting the correction from a
    lattice P reproduces P's velocity on every fluid cell (u_fine + (u(P) -
    u_fine)); accumulating a second time from the same lattice changes
    nothing further once u_fine equals u(P); mode 0 stops it."""
    n = 16
    N = 2 * n
    c, w, _ = oracle.velocity_set()
    rng = np.random.default_rng(12)
    solid = to_dev(inputs.random_mask((N, N, N), 0.1, seed=13)).reshape(N, N, N)
    feq = oracle.lbm_equilibrium(1.0, np.array([0.04, 0.0, 0.01]))
    fa = to_dev((feq[:, None] + rng.uniform(-1e-3, 1e-3, (19, N ** 3)) - w[:, None])
                .astype(np.float32).reshape(19, N, N, N))
    fp = to_dev((feq[:, None] + rng.uniform(-1e-3, 1e-3, (19, N ** 3)) - w[:, None])
                .astype(np.float32).reshape(19, N, N, N))
    s = B.Surrogate(n)
    s.set_params(torch.zeros(s.nparams, dtype=torch.float32, device="cuda"))
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")

    def err_to(f):
        sums.zero_()
        s.fine_velocity_error(f, solid, sums)
        e, r = sums.tolist()
        return (e / r) ** 0.5

    s.features(fa, solid, 20.0)
    assert err_to(fp) > 1e-2
    s.set_correction(fp, solid, 1)
    s.forward(keep_activations=False)
    s.advance_fine(1e-3, solid, 20.0)
    assert err_to(fp) <= 1e-6
    s.set_correction(fp, solid, 2)   # the defect is now zero: the correction stays
    s.features(fa, solid, 20.0)
    s.forward(keep_activations=False)
    s.advance_fine(1e-3, solid, 20.0)
    assert err_to(fp) <= 1e-6
    s.set_correction(None, None, 0)
    s.features(fa, solid, 20.0)
    s.forward(keep_activations=False)
    s.advance_fine(1e-3, solid, 20.0)
    assert err_to(fp) > 1e-2
    s.close()


def _planar_bf16(n, c, seed):
    """A random BF16 volume in the planar layout [c/8][n^3][8] (device) and
    the same values as float64 [c][z][y][x] (host)."""
    rng = np.random.default_rng(seed)
    v = torch.tensor(rng.standard_normal((c // 8, n ** 3, 8)).astype(np.float32)).to(torch.bfloat16)
    ref = v.to(torch.float64).numpy().reshape(c // 8, n, n, n, 8)
    ref = np.moveaxis(ref, 4, 1).reshape(c, n, n, n)
    return v.cuda().contiguous(), ref


@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("shape", [(16, 32), (32, 32), (32, 16)])
def test_weight_gradient_kernels_match_the_sum(n, shape):
    """surr_weight_grad, both implementations (tcgen05 with TMA-loaded MN-major
    operands, the one surr_backward runs; and the mma.sync kernel), against
    the definition dW[tap][co][ci] = sum_v g[v][co] in[v + d(tap)][ci] with
    zero padding, summed in float64 from the same BF16 values, for every layer
    shape; the bias gradient sum_v g[v][co]; a second call accumulates. Both
    sum in FP32: relative L2 2e-5 at 16^3 voxels, 1e-4 at 64^3."""
    cin, cout = shape
    x, X = _planar_bf16(n, cin, seed=cin + 7 * n)
    g, G = _planar_bf16(n, cout, seed=cout + 11 * n)
    Xp = np.pad(X, ((0, 0), (1, 1), (1, 1), (1, 1)))
    ref = np.zeros((27, cout, cin))
    Gm = G.reshape(cout, -1)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sh = Xp[:, dz:dz + n, dy:dy + n, dx:dx + n].reshape(cin, -1)
                ref[9 * dz + 3 * dy + dx] = Gm @ sh.T
    ref_b = Gm.sum(axis=1)
    tol = 2e-5 if n == 16 else 1e-4
    s = B.Surrogate(n)
    got = {}
    for impl in (0, 1):
        gw = torch.zeros(27 * cout * cin, device="cuda")
        gb = torch.zeros(cout, device="cuda")
        s.weight_grad(cin, cout, x, g, gw, gb, impl=impl)
        s.device_status()
        w = gw.double().cpu().numpy().reshape(27, cout, cin)
        assert rel_l2(w, ref) <= tol, (impl, rel_l2(w, ref))
        assert rel_l2(gb.double().cpu().numpy(), ref_b) <= tol, impl
        got[impl] = w
        s.weight_grad(cin, cout, x, g, gw, gb, impl=impl)  # accumulates
        assert rel_l2(gw.double().cpu().numpy().reshape(27, cout, cin), 2 * ref) <= tol
    assert rel_l2(got[0], got[1]) <= tol
    s.close()
