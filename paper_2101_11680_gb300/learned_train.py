"""Training and evaluation of the learned unrolled solver (``ctof.Learned``).

Training data: seeded phantoms (1-8 random ellipsoids and tubes,
``synth.phantom_shapes``) pushed through the library's forward operator and
given Poisson counting noise at a stated peak (``synth.poisson_noise``).  Each
phantom seed is used once.  Phantom rendering and noise run on a host thread
pool (NumPy releases the interpreter lock in its array loops) one batch ahead
of the GPU, so the device only runs the forward operator, the unrolled solver
and its backward pass.

Evaluation compares the learned solver with plain ADMM on the same seeded
measurements: relative volume error ||x - mu|| / ||mu|| and relative data
residual ||A x - m|| / ||m||, with ADMM as the fallback whenever the learned
residual exceeds a threshold (1.5 x the ADMM residual of a calibration set).

Usage (writes the parameter file that ``load`` reads):
    python -m paper_2101_11680_gb300.learned_train --out FILE [--phantoms 20000]
"""

import argparse
import json
import math
from multiprocessing.pool import ThreadPool
import os
import time

import numpy as np

from . import synth

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_WEIGHTS = os.path.join(WEIGHTS_DIR, "learned_s10.npz")

# Optics of the training and evaluation data (1/mm, refractive index).
OPTICS = dict(mua=0.01, musp=1.0, n=1.4)
# Evaluation geometry: 128 x 128 scan at 0.5 mm, 48 depths of 0.5 mm from 0.5 mm, 256 bins of 25 ps.
EVAL_GRID = dict(n=128, nz=48, nt=256, dx=0.5, dz=0.5, z_first=0.5, dt=25.0)
# Training geometry: the same pitches, depths and bins on a 64 x 64 lateral field.
TRAIN_GRID = dict(EVAL_GRID, n=64)
PEAK = 1e5
# Start of the unrolled stages: the per-frequency Tikhonov solution at this relative lambda.
X0_LAMBDA = 1e-3
# Inference-time data-consistency steps after the last stage and their relative Tikhonov lambda.
DC_STEPS = 3
DC_LAMBDA = 1e-5


def _render(args):
    seed, g = args
    return synth.phantom_shapes(g["n"], g["nz"], g["dx"], g["dz"], g["z_first"], seed=seed).astype(np.float32)


def _noise(args):
    clean, peak, seed = args
    return synth.poisson_noise(np.clip(clean, 0.0, None), peak, seed).astype(np.float32)


def noise_seed(seed):
    """Seed of the Poisson draw that goes with phantom ``seed``."""
    return 1_000_003 + int(seed)


def make_kernel(grid_kw):
    from . import ctof
    g = grid_kw
    return ctof.Kernel(ctof.make_optics(**OPTICS),
                       ctof.make_grid(g["n"], g["nz"], g["nt"], g["dx"], g["dz"], g["z_first"], g["dt"]))


class DataPipe:
    """Seeded (measurement, phantom) batches on the device, prepared one batch ahead."""

    def __init__(self, kernel, grid_kw, seeds, batch, peak=PEAK, workers=None):
        import torch
        self.k, self.g, self.batch, self.peak = kernel, grid_kw, batch, peak
        self.seeds = list(seeds)
        self.pos = 0
        workers = workers or max(2, min(16, (os.cpu_count() or 4) - 1))
        self.pool = ThreadPool(workers)
        self.torch = torch
        self._mu_next = self._submit_render()
        self._pending = None

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def _take_seeds(self):
        out = [self.seeds[(self.pos + i) % len(self.seeds)] for i in range(self.batch)]
        self.pos += self.batch
        return out

    def _submit_render(self):
        s = self._take_seeds()
        return s, self.pool.map_async(_render, [(x, self.g) for x in s])

    def _stage(self):
        """Clean measurements of the rendered batch on the device, noise submitted to the pool."""
        torch = self.torch
        seeds, job = self._mu_next
        mus = job.get()
        self._mu_next = self._submit_render()
        d_mu = torch.tensor(np.stack(mus), device="cuda")
        clean = torch.empty((self.batch, self.g["nt"], self.g["n"], self.g["n"]), device="cuda")
        for b in range(self.batch):
            self.k.forward(d_mu[b], out=clean[b])
        host = clean.cpu().numpy()
        return d_mu, self.pool.map_async(_noise, [(host[b], self.peak, noise_seed(s)) for b, s in enumerate(seeds)])

    def next(self):
        torch = self.torch
        if self._pending is None:
            self._pending = self._stage()
        d_mu, job = self._pending
        self._pending = self._stage()
        d_m = torch.tensor(np.stack(job.get()), device="cuda")
        return d_m, d_mu


def train(kernel, grid_kw, stages=10, phantoms=20000, batch=4, lr=1e-3, lr_final=1e-4, seed0=0, init_seed=7,
          peak=PEAK, x0_lambda_rel=X0_LAMBDA, log_every=100, log=print):
    """Adam on the mean squared volume error; cosine learning-rate decay lr -> lr_final.

    Returns (Learned handle, history [(step, loss, seconds)]).
    """
    from . import ctof
    net = ctof.Learned(stages, synth.learned_init(stages, init_seed), x0_lambda_rel)
    steps = max(1, phantoms // batch)
    pipe = DataPipe(kernel, grid_kw, range(seed0, seed0 + steps * batch), batch, peak)
    hist = []
    t0 = time.time()
    try:
        for it in range(steps):
            d_m, d_mu = pipe.next()
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / steps))
            want = (it % log_every == 0) or it == steps - 1
            loss = net.train_step(kernel, d_m, d_mu, a, want_loss=want)
            if want:
                hist.append((it, loss, time.time() - t0))
                if log:
                    log(f"step {it}/{steps} loss {loss:.5f} lr {a:.2e} {time.time() - t0:.1f}s")
    finally:
        pipe.close()
    return net, hist


def save(path, net, meta):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    meta = dict(meta, x0_lambda_rel=net.x0_lambda_rel)
    np.savez(path, theta=net.params(), stages=np.int32(net.stages), meta=np.array(json.dumps(meta)))


def load(path=DEFAULT_WEIGHTS):
    """(flat FP32 parameters, stages, metadata dict) from a file written by ``save``.

    ``metadata["x0_lambda_rel"]`` is the start the parameters were trained with.
    """
    z = np.load(path)
    return z["theta"].astype(np.float32), int(z["stages"]), json.loads(str(z["meta"]))


def make_net(theta, stages, meta, dc_steps=DC_STEPS, dc_lambda_rel=DC_LAMBDA):
    """Inference handle for trained parameters (the start they were trained with, plus data consistency)."""
    from . import ctof
    return ctof.Learned(stages, theta, meta.get("x0_lambda_rel", 0.0), dc_steps, dc_lambda_rel)


def volume_error(x, mu):
    return float((x.double() - mu.double()).norm() / mu.double().norm())


def data_residual(kernel, x, m):
    return float((kernel.forward(x).double() - m.double()).norm() / m.double().norm())


def eval_set(kernel, grid_kw, seeds, peak=PEAK):
    """Device (measurement, phantom) pairs for evaluation seeds (host-rendered, no pool)."""
    import torch
    out = []
    for s in seeds:
        mu = torch.tensor(_render((s, grid_kw)), device="cuda")
        clean = kernel.forward(mu).cpu().numpy()
        m = torch.tensor(_noise((clean, peak, noise_seed(s))), device="cuda")
        out.append((m, mu))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--stages", type=int, default=10)
    ap.add_argument("--phantoms", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lateral", type=int, default=TRAIN_GRID["n"])
    args = ap.parse_args(argv)
    from . import build
    build.build()
    g = dict(TRAIN_GRID, n=args.lateral)
    k = make_kernel(g)
    net, hist = train(k, g, stages=args.stages, phantoms=args.phantoms, batch=args.batch, lr=args.lr)
    meta = dict(grid=g, optics=OPTICS, peak=PEAK, phantoms=args.phantoms, batch=args.batch, lr=args.lr,
                seeds=[0, args.phantoms], init_seed=7, history=hist)
    save(args.out, net, meta)
    print(json.dumps(dict(out=args.out, final_loss=hist[-1][1], seconds=hist[-1][2])))


if __name__ == "__main__":
    main()
