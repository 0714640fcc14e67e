"""Learned form on the device against the FP64 oracle (``oracle.learned``).

The device runs the 3-D CNN with BF16 weights, activations and inter-layer
gradients, FP32 accumulation and FP32 master parameters.  The test weights
are put on the BF16 grid, so both sides evaluate the same network; what
remains is the rounding of stored activations and gradients (relative error
at most 2^-9 each).  Two comparisons:

* against the FP64 oracle with the same storage points rounded to BF16
  (``rnd=oracle.learned.bf16``): the device must agree to 2e-3 per parameter
  tensor and 2e-4 on the loss and the reconstruction (what is left is FP32 vs
  FP64 accumulation, and the odd element whose FP32 sum falls on the other
  side of a BF16 rounding boundary);
* against the exact FP64 oracle, which measures the roundings themselves: the
  loss to 1e-3, the whole gradient to 3e-2 and each parameter tensor to
  1.5e-2 where BF16 storage allows it.  The rounding oracle run on the CPU
  (same problems, same weights) fixes what BF16 storage alone does to each
  tensor against the exact oracle: on one problem every tensor is within
  1.14e-2 (b2 the largest); on the two-problem batch the layer-3/4 and step
  size tensors stay within 1.13e-2, while the layer-1/2 tensors are 1-21 %
  off: their gradient is a sum over all voxels (and over the two problems)
  whose terms cancel to a small fraction of their absolute sum, and
  pre-activations within a rounding error of zero switch their ReLU.  Those
  four tensors are held there by the whole-gradient bound and, per tensor,
  by the rounding oracle.
"""

import numpy as np
import pytest

from oracle import learned as ln
from oracle import operators as op
from oracle import solvers as so
from paper_2101_11680_gb300 import ctof, synth

from gpu_common import CASES, device_kernel, oracle_kernel, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASE = "admm16"  # 16 x 16 scan, 6 depths, 32 bins
STAGES = 3
TENSORS = ["w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "eta"]
# tensors held per tensor against the exact FP64 oracle, by batch size (see the module docstring)
EXACT_PER_TENSOR = {1: set(TENSORS), 2: {"w3", "b3", "w4", "b4", "eta"}}


def _problem(seed):
    kw = CASES[CASE]
    g, _, wh = oracle_kernel(CASE)
    mu = synth.phantom_shapes(kw["n"], kw["nz"], kw["dx"], kw["dz"], kw["z_first"], seed=seed, max_shapes=4)
    m = synth.poisson_noise(np.clip(op.forward_fft(wh, mu, g), 0.0, None), 1e5, seed=seed + 1)
    return mu, m


def _params(seed):
    theta = synth.learned_init(STAGES, seed)
    rng = np.random.default_rng(seed)
    # non-zero biases and step sizes away from 1 so that every term is exercised
    off = 0
    for ci, co in synth.LEARNED_LAYERS:
        off += co * ci * 27
        theta[off:off + co] = rng.normal(0.0, 0.05, co)
        off += co
    theta[-STAGES:] = rng.uniform(0.7, 1.3, STAGES)
    return theta


def _on_bf16_grid(theta):
    """Weights rounded to BF16 (biases and step sizes stay FP32 on the device)."""
    theta = theta.copy()
    off = 0
    for ci, co in synth.LEARNED_LAYERS:
        theta[off:off + co * ci * 27] = ln.bf16(theta[off:off + co * ci * 27])
        off += co * ci * 27 + co
    return theta


def _oracle_ops():
    g, _, wh = oracle_kernel(CASE)
    s = so.spectral_norm(wh)
    return (lambda v: op.forward_fft(wh / s, v, g)), (lambda r: op.adjoint_fft(wh / s, r, g)), s


def _tensors(flat):
    layers, eta = ln.unpack(flat, STAGES)
    out = []
    for w, b in layers:
        out += [w, b]
    return out + [eta]


def test_learned_loss_and_gradient_match_oracle():
    k = device_kernel(CASE)
    fwd, adj, s = _oracle_ops()
    theta = _on_bf16_grid(_params(21))
    net = ctof.Learned(STAGES, theta)
    for batch in (1, 2):
        probs = [_problem(300 + i) for i in range(batch)]
        d_m = torch.tensor(np.stack([m for _, m in probs]), dtype=torch.float32, device="cuda")
        d_mu = torch.tensor(np.stack([mu for mu, _ in probs]), dtype=torch.float32, device="cuda")
        got_l, got_g = net.loss_grad(k, d_m, d_mu)
        for rnd in (ln.bf16, None):
            want_l, want_g = 0.0, np.zeros_like(theta)
            for mu, m in probs:
                l, gr = ln.loss_and_grad(theta, STAGES, fwd, adj, m / s, mu, rnd=rnd)
                want_l += l / batch
                want_g += gr / batch
            if rnd is not None:
                assert got_l == pytest.approx(want_l, rel=2e-4)
                for name, gt, wt in zip(TENSORS, _tensors(got_g), _tensors(want_g)):
                    assert rel_l2(gt, wt) <= 2e-3, (batch, name, rel_l2(gt, wt))
            else:
                assert got_l == pytest.approx(want_l, rel=1e-3)
                assert rel_l2(got_g, want_g) <= 3e-2
                exact_ok = EXACT_PER_TENSOR[batch]
                for name, gt, wt in zip(TENSORS, _tensors(got_g), _tensors(want_g)):
                    if name in exact_ok:
                        assert rel_l2(gt, wt) <= 1.5e-2, (batch, name, rel_l2(gt, wt))
    net.close()


def test_learned_tikhonov_start_matches_oracle():
    """x_0 = the per-frequency Tikhonov solution (lambda 1e-3 max Gram diagonal).

    The device's x_0 carries the FP32 Tikhonov solve's own error (1e-5
    relative, that solver's parity bound), which moves a few stored values
    across BF16 rounding boundaries.  Small, cancelling tensors (a bias
    gradient whose entries are sums of terms of both signs) feel that most, so
    here the whole gradient is held to 2e-3, each tensor to 2e-2 and the
    reconstruction to 2e-3 (measured: 4.6e-4); the zero start holds every
    tensor to 2e-3 and the reconstruction to 2e-4.
    """
    k = device_kernel(CASE)
    fwd, adj, s = _oracle_ops()
    g, _, wh = oracle_kernel(CASE)
    theta = _on_bf16_grid(_params(25))
    net = ctof.Learned(STAGES, theta, x0_lambda_rel=1e-3)
    probs = [_problem(600 + i) for i in range(2)]
    d_m = torch.tensor(np.stack([m for _, m in probs]), dtype=torch.float32, device="cuda")
    d_mu = torch.tensor(np.stack([mu for mu, _ in probs]), dtype=torch.float32, device="cuda")
    got_l, got_g = net.loss_grad(k, d_m, d_mu)
    want_l, want_g, want_x = 0.0, np.zeros_like(theta), []
    for mu, m in probs:
        x0 = so.tikhonov(wh, m, g, 1e-3)[0]
        l, gr = ln.loss_and_grad(theta, STAGES, fwd, adj, m / s, mu, rnd=ln.bf16, x0=x0)
        want_l += l / 2
        want_g += gr / 2
        want_x.append(ln.unrolled(theta, STAGES, fwd, adj, m / s, rnd=ln.bf16, x0=x0))
    assert got_l == pytest.approx(want_l, rel=2e-4)
    assert rel_l2(got_g, want_g) <= 2e-3
    for name, gt, wt in zip(["w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "eta"], _tensors(got_g), _tensors(want_g)):
        assert rel_l2(gt, wt) <= 2e-2, (name, rel_l2(gt, wt))
    got_x = net.reconstruct(k, d_m).cpu().numpy()
    assert rel_l2(got_x, np.stack(want_x)) <= 2e-3
    net.close()


def test_learned_data_consistency_steps_match_oracle():
    k = device_kernel(CASE)
    fwd, adj, s = _oracle_ops()
    g, _, wh = oracle_kernel(CASE)
    theta = _on_bf16_grid(_params(26))
    net = ctof.Learned(STAGES, theta, x0_lambda_rel=1e-3, dc_steps=2, dc_lambda_rel=1e-4)
    mu, m = _problem(700)
    x0 = so.tikhonov(wh, m, g, 1e-3)[0]
    tik = lambda r: so.tikhonov(wh / s, r, g, 1e-4)[0]
    want = ln.unrolled(theta, STAGES, fwd, adj, m / s, rnd=ln.bf16, x0=x0, dc_steps=2, dc_solve=tik)
    got = net.reconstruct(k, torch.tensor(m[None], dtype=torch.float32, device="cuda"))[0].cpu().numpy()
    assert rel_l2(got, want) <= 2e-3
    # the steps pull the result towards the data
    plain = ln.unrolled(theta, STAGES, fwd, adj, m / s, rnd=ln.bf16, x0=x0)
    assert np.linalg.norm(fwd(got) - m / s) < np.linalg.norm(fwd(plain) - m / s)
    net.close()


def test_learned_batch_of_five_matches_oracle():
    """A batch of five volumes takes the batched tensor-core contractions (forward,
    adjoint, and the Tikhonov start / data-consistency solves: adjoint on tcgen05
    plus the per-class inverse); every member still matches the FP64 oracle run
    on it alone, at the bound of the single-volume Tikhonov-start test."""
    k = device_kernel(CASE)
    fwd, adj, s = _oracle_ops()
    g, _, wh = oracle_kernel(CASE)
    theta = _on_bf16_grid(_params(27))
    net = ctof.Learned(STAGES, theta, x0_lambda_rel=1e-3, dc_steps=2, dc_lambda_rel=1e-4)
    probs = [_problem(800 + i) for i in range(5)]
    d_m = torch.tensor(np.stack([m for _, m in probs]), dtype=torch.float32, device="cuda")
    got = net.reconstruct(k, d_m).cpu().numpy()
    tik = lambda r: so.tikhonov(wh / s, r, g, 1e-4)[0]
    for b, (mu, m) in enumerate(probs):
        x0 = so.tikhonov(wh, m, g, 1e-3)[0]
        want = ln.unrolled(theta, STAGES, fwd, adj, m / s, rnd=ln.bf16, x0=x0, dc_steps=2, dc_solve=tik)
        assert rel_l2(got[b], want) <= 2e-3, b
    net.close()


@pytest.mark.parametrize("batch", [1, 5])
def test_learned_reconstruct_checked_residuals(batch):
    """ctof_learned_reconstruct_checked: the volumes equal ctof_learned_reconstruct's,
    and each member's ||A mu - m|| / ||m|| matches the FP64 oracle's forward operator
    (Eq. 11) applied to the returned volume, to 1e-4 relative (the device forms
    A mu in FP32; the residual is a tenth of ||m|| or more, so its FP32 error stays
    near 1e-5).  An all-zero measurement gives +inf when the oracle's A mu is
    non-zero (the network's biases make it so)."""
    k = device_kernel(CASE)
    g, _, wh = oracle_kernel(CASE)
    theta = _on_bf16_grid(_params(28))
    net = ctof.Learned(STAGES, theta, x0_lambda_rel=1e-3, dc_steps=1, dc_lambda_rel=1e-4)
    ms = [_problem(900 + i)[1] for i in range(batch)]
    if batch > 1:
        ms[-1] = np.zeros_like(ms[-1])
    d_m = torch.tensor(np.stack(ms), dtype=torch.float32, device="cuda")
    plain = net.reconstruct(k, d_m)
    got, res = net.reconstruct_checked(k, d_m)
    torch.cuda.synchronize()
    assert torch.equal(got, plain)
    x = got.cpu().numpy().astype(np.float64)
    res = res.cpu().numpy()
    for b, m in enumerate(ms):
        r = np.linalg.norm(op.forward_fft(wh, x[b], g) - m)
        if np.linalg.norm(m) == 0.0:
            assert r > 0.0 and np.isinf(res[b]), (b, res[b])
        else:
            want = r / np.linalg.norm(m)
            assert abs(res[b] - want) <= 1e-4 * want, (b, res[b], want)
    with pytest.raises(TypeError):
        net.reconstruct_checked(k, d_m, res=torch.empty(batch, device="cuda", dtype=torch.float32))
    net.close()


def test_learned_full_width_rows_match_oracle():
    """Scan rows of 128 voxels fill the convolution's 128-row tensor-core tile
    exactly (x - 1 and x + 128 from the zero padding), 128 rows make four row
    bands, 4 depths put every plane next to a border: a batch of four (the
    batched tensor-core contractions and the plane-batched depth FFTs) through the
    Tikhonov start, two stages and one data-consistency step matches the FP64
    oracle with BF16 storage points to 2e-3 per member, as at the small sizes."""
    case = "wide128"
    kw = CASES[case]
    k = device_kernel(case)
    g, _, wh = oracle_kernel(case)
    s = so.spectral_norm(wh)
    fwd = lambda v: op.forward_fft(wh / s, v, g)
    adj = lambda r: op.adjoint_fft(wh / s, r, g)
    stages = 2
    theta = synth.learned_init(stages, 31)
    rng = np.random.default_rng(31)
    off = 0
    for ci, co in synth.LEARNED_LAYERS:
        theta[off:off + co * ci * 27] = ln.bf16(theta[off:off + co * ci * 27])
        off += co * ci * 27
        theta[off:off + co] = rng.normal(0.0, 0.05, co)
        off += co
    theta[-stages:] = rng.uniform(0.7, 1.3, stages)
    net = ctof.Learned(stages, theta, x0_lambda_rel=1e-3, dc_steps=1, dc_lambda_rel=1e-4)
    ms = []
    for i in range(4):
        mu = synth.phantom_shapes(kw["n"], kw["nz"], kw["dx"], kw["dz"], kw["z_first"], seed=950 + i, max_shapes=6)
        ms.append(synth.poisson_noise(np.clip(op.forward_fft(wh, mu, g), 0.0, None), 1e5, seed=960 + i))
    got = net.reconstruct(k, torch.tensor(np.stack(ms), dtype=torch.float32, device="cuda")).cpu().numpy()
    tik = lambda r: so.tikhonov(wh / s, r, g, 1e-4)[0]
    for b, m in enumerate(ms):
        x0 = so.tikhonov(wh, m, g, 1e-3)[0]
        want = ln.unrolled(theta, stages, fwd, adj, m / s, rnd=ln.bf16, x0=x0, dc_steps=1, dc_solve=tik)
        assert rel_l2(got[b], want) <= 2e-3, (b, rel_l2(got[b], want))
    net.close()


def test_trained_network_gains_over_untrained_and_admm():
    """The shipped parameters, on held-out seeded phantoms at the training geometry
    (64 x 64 scan at 0.5 mm, 48 depths, 256 bins of 25 ps, Poisson peak 1e5): the
    trained solver's volume error is below the same solver with its initial
    parameters and below 100 iterations of plain ADMM, and the data-consistency
    steps keep its data residual at most 1.5x ADMM's on average."""
    from paper_2101_11680_gb300 import learned_train as LT
    theta, stages, meta = LT.load()
    k = LT.make_kernel(LT.TRAIN_GRID)
    data = LT.eval_set(k, LT.TRAIN_GRID, range(10000, 10006))
    trained = LT.make_net(theta, stages, meta)
    untrained = LT.make_net(synth.learned_init(stages, 7).astype(np.float32), stages, meta)
    p = ctof.admm_params(iters=100)
    e_t, e_u, e_a, r_t, r_a = [], [], [], [], []
    for m, mu in data:
        xt = trained.reconstruct(k, m[None])[0]
        xu = untrained.reconstruct(k, m[None])[0]
        xa = k.reconstruct(m, p)
        e_t.append(LT.volume_error(xt, mu))
        e_u.append(LT.volume_error(xu, mu))
        e_a.append(LT.volume_error(xa, mu))
        r_t.append(LT.data_residual(k, xt, m))
        r_a.append(LT.data_residual(k, xa, m))
    assert np.mean(e_t) < np.mean(e_u) - 0.05
    assert np.mean(e_t) < np.mean(e_a) - 0.05
    assert np.mean(r_t) <= 1.5 * np.mean(r_a)
    trained.close()
    untrained.close()
    k.close()


def test_learned_reconstruct_matches_oracle():
    k = device_kernel(CASE)
    fwd, adj, s = _oracle_ops()
    theta = _on_bf16_grid(_params(22))
    net = ctof.Learned(STAGES, theta)
    mu, m = _problem(400)
    got = net.reconstruct(k, torch.tensor(m[None], dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rel_l2(got[0].cpu().numpy(), ln.unrolled(theta, STAGES, fwd, adj, m / s, rnd=ln.bf16)) <= 2e-4
    assert rel_l2(got[0].cpu().numpy(), ln.unrolled(theta, STAGES, fwd, adj, m / s)) <= 5e-3
    # reproducible
    got2 = net.reconstruct(k, torch.tensor(m[None], dtype=torch.float32, device="cuda"))
    assert torch.equal(got, got2)
    net.close()


def test_learned_params_roundtrip_and_validation():
    k = device_kernel(CASE)
    theta = _params(23)
    net = ctof.Learned(STAGES, theta)
    assert np.array_equal(net.params(), theta.astype(np.float32))
    # lateral size not a multiple of 16 is refused
    k12 = device_kernel("aniso")
    with pytest.raises(ctof.CtofError):
        net.reconstruct(k12, torch.zeros((1, 10, 12, 12), device="cuda"))
    net.close()


def test_learned_train_step_descends():
    k = device_kernel(CASE)
    theta = _params(24)
    net = ctof.Learned(STAGES, theta)
    probs = [_problem(500 + i) for i in range(2)]
    d_m = torch.tensor(np.stack([m for _, m in probs]), dtype=torch.float32, device="cuda")
    d_mu = torch.tensor(np.stack([mu for mu, _ in probs]), dtype=torch.float32, device="cuda")
    l0 = net.loss_grad(k, d_m, d_mu)[0]
    for _ in range(30):
        net.train_step(k, d_m, d_mu, 1e-3)
    l1 = net.loss_grad(k, d_m, d_mu)[0]
    assert l1 < 0.9 * l0
    assert np.all(np.isfinite(net.params()))
    net.close()
