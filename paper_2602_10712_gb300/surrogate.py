"""The neural proxy of Sec. 3.3 trained on data the tracer generates.

Design space (16 parameters, the box-wing with 7 material groups): rho_s and
rho_d of the 6 bus faces and the panels (14 values in [0, 0.5]) and the two
panel hinge angles (in [-pi/2, pi/2]); inputs are the body-frame sun
direction (3) and the scaled design vector (16).  Outputs: force and torque
for unit radiation pressure, standardised per component.

Everything numeric runs in the library's kernels: design instantiation and
BVH build (host C++), srp_force (tracer), srp_mlp_train_step / srp_mlp_infer
(tensor-core MLP).  This module only orchestrates them.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import MLP, Context, srp_build_bvh, srp_design_instantiate, srp_force

N_DESIGN = 16
HINGE_MAX = math.pi / 2
RHO_MAX = 0.5   # the training range of every reflectance: [0, RHO_MAX]


def sample_designs(n: int, seed: int) -> np.ndarray:
    """theta [n,16]: rho_s[7], rho_d[7] ~ U[0,0.5], hinge[2] ~ U[-pi/2, pi/2]."""
    rng = np.random.default_rng(seed)
    th = np.empty((n, N_DESIGN))
    th[:, :14] = rng.uniform(0.0, RHO_MAX, size=(n, 14))
    th[:, 14:] = rng.uniform(-HINGE_MAX, HINGE_MAX, size=(n, 2))
    return th


def sample_suns(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def encode(sun: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Network input [.,19]: sun (3), 4*rho - 1 (14), hinge / (pi/2) (2)."""
    x = np.empty(sun.shape[:-1] + (19,), np.float32)
    x[..., :3] = sun
    x[..., 3:17] = 4.0 * theta[..., :14] - 1.0
    x[..., 17:] = theta[..., 14:] / HINGE_MAX
    return x


def trace_dataset(ctx: Context, mesh, theta: np.ndarray, suns_per_design: int, rays: int, bounces: int,
                  seed: int, sun_seed: int):
    """MC force/torque for every (design, sun): (sun [D,S,3], ft [D,S,6])."""
    D = theta.shape[0]
    sun = sample_suns(D * suns_per_design, sun_seed).reshape(D, suns_per_design, 3)
    rho = np.zeros((D, mesh.n_groups, 2), np.float32)
    rho[:, :, 0] = theta[:, :7]
    rho[:, :, 1] = theta[:, 7:14]
    com = np.zeros((D, 3))
    ft = np.zeros((D, suns_per_design, 6))
    chunk = 512
    for d0 in range(0, D, chunk):
        d1 = min(D, d0 + chunk)
        bvhs = []
        for d in range(d0, d1):
            v = srp_design_instantiate(mesh.verts, mesh.vhinge, mesh.hinges, theta[d, 14:])
            bvhs.append(srp_build_bvh(ctx, v, mesh.tris, mesh.group, 4))
        ft[d0:d1] = srp_force(ctx, bvhs, rho[d0:d1], sun[d0:d1], com[d0:d1], rays_x=rays, max_bounces=bounces,
                              seed=seed, sun_per_design=1, design_base=d0)
        for b in bvhs:
            b.close()
    return sun, ft


class Surrogate:
    """A trained proxy: MLP + output standardisation."""

    def __init__(self, ctx: Context, net: MLP, mean: np.ndarray, std: np.ndarray):
        self.ctx, self.net, self.mean, self.std = ctx, net, mean, std

    def predict(self, sun: np.ndarray, theta: np.ndarray) -> np.ndarray:
        x = encode(sun, theta).reshape(-1, 19)
        y = self.net.infer(x)
        return y.astype(np.float64) * self.std + self.mean

    @staticmethod
    def in_domain(theta: np.ndarray) -> np.ndarray:
        """Rows of theta [N,16] inside the training domain (reflectances in
        [0, 0.5], hinge angles in [-pi/2, pi/2])."""
        th = np.asarray(theta, np.float64).reshape(-1, N_DESIGN)
        return (np.all((th[:, :14] >= 0.0) & (th[:, :14] <= RHO_MAX), axis=1) &
                np.all(np.abs(th[:, 14:]) <= HINGE_MAX, axis=1))

    def evaluate(self, sun: np.ndarray, theta: np.ndarray, mesh, rays: int = 256, bounces: int = 3, seed: int = 0):
        """Force and torque [N,6] for unit radiation at each row (sun [N,3],
        theta [N,16]): the proxy where the design lies in its training
        domain, the ray tracer (design instantiated, BVH built, srp_force
        with rays^2 rays and up to `bounces` bounces) where it does not --
        the tracer is the proxy's fallback outside the data it was fitted
        to.  Returns (ft [N,6], traced [N] bool)."""
        sun = np.asarray(sun, np.float64).reshape(-1, 3)
        theta = np.asarray(theta, np.float64).reshape(-1, N_DESIGN)
        ok = self.in_domain(theta)
        ft = np.zeros((sun.shape[0], 6))
        if ok.any():
            ft[ok] = self.predict(sun[ok], theta[ok])
        for i in np.flatnonzero(~ok):
            v = srp_design_instantiate(mesh.verts, mesh.vhinge, mesh.hinges, theta[i, 14:])
            b = srp_build_bvh(self.ctx, v, mesh.tris, mesh.group, 4)
            rho = np.stack([theta[i, :7], theta[i, 7:14]], axis=1).astype(np.float32)[None]
            ft[i] = srp_force(self.ctx, [b], rho, sun[i:i + 1], np.zeros((1, 3)), rays_x=rays, max_bounces=bounces,
                              seed=seed, sun_base=int(i))[0, 0]
            b.close()
        return ft, ~ok


def fit(ctx: Context, mesh, n_designs=4096, suns_per_design=256, rays=256, bounces=3, epochs=20, batch=8192,
        lr=2e-3, seed=0, log=None, checkpoint=None, resume=False, device=None):
    """Generate the data with the tracer and train the proxy; returns
    (Surrogate, info dict with timings).

    checkpoint: a path prefix; after every epoch the network's trainer state
    (parameters, Adam moments, step: <prefix>.state, srp_mlp_save_state) and
    the loop's own state (epochs done, step, the batch-permutation RNG and
    the output standardisation: <prefix>.npz) are written, each through a
    temporary file and a rename.  resume=True continues from them when they
    exist: the data set is traced again from the same seeds (the tracer is
    deterministic), the finished epochs are skipped and the learning-rate
    schedule and batch order continue where they stopped.  device: where
    the training batches live (default: the context's GPU).  On a GPU each
    epoch is one srp_mlp_train_epoch call over a batch order drawn on the
    device from (seed, epoch); elsewhere (a stand-in network) one
    train_step per batch over a host permutation."""
    import json
    import os

    t0 = time.perf_counter()
    theta = sample_designs(n_designs, seed)
    sun, ft = trace_dataset(ctx, mesh, theta, suns_per_design, rays, bounces, seed=seed, sun_seed=seed + 1)
    t_data = time.perf_counter() - t0
    x = encode(sun, theta[:, None, :].repeat(suns_per_design, axis=1)).reshape(-1, 19)
    y = ft.reshape(-1, 6)
    mean = y.mean(axis=0)
    std = y.std(axis=0) + 1e-12
    yn = ((y - mean) / std).astype(np.float32)
    net = MLP(ctx, seed=seed)
    n = x.shape[0]
    rng = np.random.default_rng(seed + 7)
    steps = max(1, epochs * (n // batch))
    step, ep0 = 0, 0
    if resume and checkpoint is not None and os.path.exists(checkpoint + ".npz"):
        meta = np.load(checkpoint + ".npz", allow_pickle=False)
        if not (np.array_equal(meta["mean"], mean) and np.array_equal(meta["std"], std)):
            raise ValueError("checkpoint was written for another data set")
        ep0, step = int(meta["epoch"]), int(meta["step"])
        rng.bit_generator.state = json.loads(str(meta["rng"]))
        net.load_state(checkpoint + ".state")
    t1 = time.perf_counter()
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", ctx.device)
    xt = torch.from_numpy(x).to(dev)
    yt = torch.from_numpy(yn).to(dev)
    nb = n // batch
    for ep in range(ep0, epochs):
        lrs = [lr * 0.5 * (1.0 + math.cos(math.pi * (step + k) / steps)) + 1e-5 for k in range(nb)]
        if dev.type == "cuda":
            # the epoch's batch order is drawn on the device from (seed,
            # epoch) alone, so a resumed run repeats it; the batches are
            # gathered inside the training kernels and the steps queued by
            # one library call (no host round trip per step)
            g = torch.Generator(device=dev)
            g.manual_seed((seed + 7) * 1000003 + ep)
            perm = torch.randperm(n, generator=g, device=dev)[:nb * batch].to(torch.int32)
            net.train_epoch(xt, yt, perm, batch, np.array(lrs, np.float32))
        else:
            pt = torch.from_numpy(rng.permutation(n)).to(dev)
            for k in range(nb):
                idx = pt[k * batch:(k + 1) * batch]
                net.train_step(xt.index_select(0, idx).contiguous(), yt.index_select(0, idx).contiguous(), lrs[k],
                               want_loss=False)
        step += nb
        if log is not None:
            l, _ = net.train_step(xt[:batch].contiguous(), yt[:batch].contiguous(), 0.0)
            log(f"epoch {ep} loss {l:.4f}")
        if checkpoint is not None:
            net.save_state(checkpoint + ".state.tmp")
            os.replace(checkpoint + ".state.tmp", checkpoint + ".state")
            with open(checkpoint + ".tmp.npz", "wb") as f:
                np.savez(f, epoch=ep + 1, step=step, rng=json.dumps(rng.bit_generator.state), mean=mean, std=std)
            os.replace(checkpoint + ".tmp.npz", checkpoint + ".npz")
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t1
    return Surrogate(ctx, net, mean, std), {"data_s": t_data, "train_s": t_train, "samples": n, "steps": step}


def force_rms_error(sur: Surrogate, ctx: Context, mesh, n_designs=256, suns_per_design=16, rays=1024, bounces=3,
                    seed=99):
    """sqrt(mean |F_nn - F_mc|^2) / sqrt(mean |F_mc|^2) on held-out designs
    and directions, F_mc traced with `rays`^2 rays (16x the training rays
    by default)."""
    theta = sample_designs(n_designs, seed)
    sun, ft = trace_dataset(ctx, mesh, theta, suns_per_design, rays, bounces, seed=seed, sun_seed=seed + 1)
    pred = sur.predict(sun, theta[:, None, :].repeat(suns_per_design, axis=1)).reshape(ft.shape)
    num = np.sqrt(np.mean(np.sum((pred[..., :3] - ft[..., :3]) ** 2, axis=-1)))
    den = np.sqrt(np.mean(np.sum(ft[..., :3] ** 2, axis=-1)))
    return num / den
