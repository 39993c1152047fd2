"""Learned warm start: a network predicts the equilibrated state of a film
with capsules from its set-up, so that the coupled run starts near
equilibrium instead of from the flat film.

Two networks run on the library's CUDA kernels:
- the 3-D U-net of unet.py (1.44M parameters, tensor-core convolutions) that
  the library's cf_warmstart runs: density corrections and node
  displacements, trained on capsule pairs of the sweep's generator
  (pair_dataset, train_unet) and measured by the time to a 1% lateral force
  (time_to_force);
- WarmNet below, the first, smaller form (five dilated 3x3x3 convolutions
  4 -> 16 -> 16 -> 16 -> 16 -> 2, dilations 1, 2, 4, 8, 1, on the FP32
  layer kernels cf_conv3d_forward / cf_conv3d_backward / cf_mse / cf_adam),
  kept with its set-up path (warm_start) and its convergence study.

Inputs per lattice node:
  0  capsule interior (1 inside a membrane, from the cut links)
  1  phi of the flat initial film, phi = (rho_A - rho_B) / (rho_maj - rho_min)
  2  z / nz
  3  log10(kS) + 2 (shear modulus of the capsule)
Density outputs: the equilibrium corrections of both densities on fluid
nodes, (rho_c,eq - rho_c,film) / (rho_maj - rho_min) for c = A, B.  The
predicted state is the film plus these corrections outside the capsules (at
least 1e-3), the film values inside; each component is then scaled on the
fluid outside the capsules to the flat film's mass, which the run conserves.

The warm-started run judges its own start: it advances two short windows and
falls back to the flat film when densities turn non-finite or negative, a
velocity exceeds a low-Mach limit, or the density change of the second window
exceeds 1.5 times that of the first (the residual grows instead of decaying).

The inputs (cf_warm_features), the predicted state with its mass matching
(cf_warm_apply), the training targets (cf_warm_target) and the residual
statistics (cf_field_check) are computed by the library's kernels too.
"""
import ctypes as C
import math

import numpy as np

from . import capfilm as cfm
from . import inputs as I

LAYERS = [(4, 16, 1, True), (16, 16, 2, True), (16, 16, 4, True), (16, 16, 8, True), (16, 2, 1, False)]
N_IN, N_OUT = 4, 2
D_RHO = I.RHO_MAJ - I.RHO_MIN  # scale of the outputs


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def features_dev(sim, wl):
    """Network inputs [4][N] and fluid mask [N] of lattice wl as float32 device
    tensors, computed by cf_warm_features."""
    import torch
    x = torch.empty(N_IN * sim.N, dtype=torch.float32, device="cuda")
    mask = torch.empty(sim.N, dtype=torch.float32, device="cuda")
    ks = wl.capsules[0].kS if wl.capsules else 1e-2
    sim.warm_features(wl.h_top, ks, x, mask)
    return x, mask


def features(sim, wl):
    """The same as host arrays [4][nz][ny][nx] and [nz][ny][nx] (training sets)."""
    x, mask = features_dev(sim, wl)
    return (x.cpu().numpy().reshape(N_IN, wl.nz, wl.ny, wl.nx),
            mask.cpu().numpy().reshape(wl.nz, wl.ny, wl.nx))


def target_of(sim, wl):
    """Network target [2][nz][ny][nx] of the current (equilibrated) state: the
    density corrections from the flat film on the fluid (cf_warm_target)."""
    import torch
    t = torch.empty(N_OUT * sim.N, dtype=torch.float32, device="cuda")
    sim.warm_target(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, t)
    return t.cpu().numpy().reshape(N_OUT, wl.nz, wl.ny, wl.nx)


class WarmNet:
    """The network's parameters and buffers on the GPU (torch tensors)."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.dev = device
        rng = np.random.default_rng(seed)
        self.w, self.b, self.wb = [], [], []
        for cin, cout, dil, relu in LAYERS:
            std = math.sqrt(2.0 / (27 * cin)) if relu else math.sqrt(1.0 / (27 * cin))
            w = rng.standard_normal((cout, cin, 27)).astype(np.float32) * std
            if not relu:
                w *= 0.1
            self.w.append(torch.from_numpy(w).to(device))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=device))
            self.wb.append(torch.empty(cout * cin * 27, dtype=torch.bfloat16, device=device))
        self.stream = torch.cuda.current_stream().cuda_stream
        self._sync_bf16()
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.t = 0

    @property
    def n_params(self):
        return sum(w.numel() + b.numel() for w, b in zip(self.w, self.b))

    def _sync_bf16(self):
        L = cfm.load_library()
        for w, wb in zip(self.w, self.wb):
            cfm._check(L.cf_to_bf16(_p(w), _p(wb), w.numel(), C.c_void_p(self.stream)))

    def to_bf16(self, a):
        torch = self.torch
        t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(self.dev)
        out = torch.empty(t.numel(), dtype=torch.bfloat16, device=self.dev)
        cfm._check(cfm._lib.cf_to_bf16(_p(t), _p(out), t.numel(), C.c_void_p(self.stream)))
        return out

    def forward(self, xb, shape):
        """xb: bfloat16 device tensor [n][4][nz][ny][nx] (flat); returns the
        activations of every layer (bfloat16, flat) with the input first."""
        torch = self.torch
        n, nz, ny, nx = shape
        acts = [xb]
        for (cin, cout, dil, relu), wb, b in zip(LAYERS, self.wb, self.b):
            y = torch.empty(n * cout * nz * ny * nx, dtype=torch.bfloat16, device=self.dev)
            cfm._check(cfm._lib.cf_conv3d_forward(_p(acts[-1]), n, cin, nz, ny, nx, _p(wb), _p(b), cout,
                                                  dil, int(relu), _p(y), C.c_void_p(self.stream)))
            acts.append(y)
        return acts

    def predict_dev(self, x, shape):
        """Density corrections for one lattice of shape (nz, ny, nx) from
        device inputs x [4][N] (float32): a float32 device tensor [2][N]."""
        torch = self.torch
        n_nodes = x.numel() // N_IN
        xb = torch.empty(x.numel(), dtype=torch.bfloat16, device=self.dev)
        cfm._check(cfm._lib.cf_to_bf16(_p(x), _p(xb), x.numel(), C.c_void_p(self.stream)))
        acts = self.forward(xb, (1,) + tuple(shape))
        out = torch.empty(N_OUT * n_nodes, dtype=torch.float32, device=self.dev)
        cfm._check(cfm._lib.cf_from_bf16(_p(acts[-1]), _p(out), out.numel(), C.c_void_p(self.stream)))
        # the simulation reads the prediction on its own stream
        torch.cuda.synchronize()
        return out

    def predict(self, x):
        """Density corrections for one lattice: x [4][nz][ny][nx] -> [2][nz][ny][nx] float32."""
        torch = self.torch
        nz, ny, nx = x.shape[1:]
        acts = self.forward(self.to_bf16(x), (1, nz, ny, nx))
        out = torch.empty(N_OUT * nz * ny * nx, dtype=torch.float32, device=self.dev)
        cfm._check(cfm._lib.cf_from_bf16(_p(acts[-1]), _p(out), out.numel(), C.c_void_p(self.stream)))
        return out.cpu().numpy().reshape(N_OUT, nz, ny, nx)

    def train_step(self, xb, target, mask, shape, lr):
        """One Adam step on a batch: xb bfloat16 inputs, target / mask float
        device tensors [n][2][nz][ny][nx]; returns the loss (masked MSE).  Each
        layer's input gradient is taken with its weights before they move."""
        torch = self.torch
        L = cfm._lib
        st = C.c_void_p(self.stream)
        n, nz, ny, nx = shape
        acts = self.forward(xb, shape)
        m = n * LAYERS[-1][1] * nz * ny * nx  # every output of the last layer
        assert target.numel() == m and mask.numel() == m
        g = torch.empty(m, dtype=torch.float32, device=self.dev)
        loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        msum = float(mask.sum().item())
        cfm._check(L.cf_mse(_p(acts[-1]), _p(target), _p(mask), m, msum, _p(g), _p(loss), st))
        self.t += 1
        for k in reversed(range(len(LAYERS))):
            cin, cout, dil, relu = LAYERS[k]
            gw = torch.zeros_like(self.w[k])
            gb = torch.zeros_like(self.b[k])
            gx = torch.empty(n * cin * nz * ny * nx, dtype=torch.float32, device=self.dev) if k > 0 else None
            cfm._check(L.cf_conv3d_backward(_p(acts[k]), n, cin, nz, ny, nx, _p(self.wb[k]), cout, dil,
                                            _p(acts[k + 1]), int(relu), _p(g), _p(gx), _p(gw), _p(gb), st))
            cfm._check(L.cf_adam(_p(self.w[k]), _p(self.wb[k]), _p(gw), _p(self.mw[k]), _p(self.vw[k]),
                                 self.w[k].numel(), lr, 0.9, 0.999, 1e-8, self.t, st))
            cfm._check(L.cf_adam(_p(self.b[k]), None, _p(gb), _p(self.mb[k]), _p(self.vb[k]),
                                 self.b[k].numel(), lr, 0.9, 0.999, 1e-8, self.t, st))
            g = gx
        return float(loss.item())

    def state(self):
        out = {f"w{k}": w.cpu().numpy() for k, w in enumerate(self.w)}
        out.update({f"b{k}": b.cpu().numpy() for k, b in enumerate(self.b)})
        return out

    def load(self, st):
        torch = self.torch
        for k in range(len(LAYERS)):
            self.w[k].copy_(torch.from_numpy(st[f"w{k}"]))
            self.b[k].copy_(torch.from_numpy(st[f"b{k}"]))
        self._sync_bf16()


def equilibrate(wls, steps, tile=1, zchunk=1):
    """Plain runs of the lattices (one batch) for `steps` steps; returns the
    simulations (with their final state)."""
    sims = [cfm.Simulation.from_workload(w) for w in wls]
    batch = cfm.Batch(sims)
    batch.set_config(tile, zchunk)
    batch.step(steps)
    batch.close()
    return sims


def dataset(wls, steps):
    """(inputs, targets, masks) of equilibrated lattices generated by the method."""
    sims = equilibrate(wls, steps)
    xs, ts, ms = [], [], []
    for s, w in zip(sims, wls):
        x, mask = features(s, w)
        xs.append(x)
        ts.append(target_of(s, w))
        ms.append(np.stack([mask] * N_OUT))
        s.close()
    return np.stack(xs), np.stack(ts), np.stack(ms)


def train(net, X, T, M, steps=300, batch=8, lr=2e-3, seed=0, log=None):
    """Adam on mini-batches drawn from the training arrays; returns the losses."""
    torch = net.torch
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    shape_v = X.shape[2:]
    losses = []
    for it in range(steps):
        idx = rng.choice(n, size=min(batch, n), replace=False)
        xb = net.to_bf16(X[idx])
        t = torch.from_numpy(np.ascontiguousarray(T[idx], np.float32)).to(net.dev).reshape(-1)
        m = torch.from_numpy(np.ascontiguousarray(M[idx], np.float32)).to(net.dev).reshape(-1)
        loss = net.train_step(xb, t, m, (len(idx),) + shape_v, lr)
        losses.append(loss)
        if log and it % 50 == 0:
            log(f"step {it}: loss {loss:.4e}")
    return losses


def warm_start(sim, wl, net, window=25, u_limit=0.1, grow=1.5):
    """Set the predicted state and judge it over two windows of `window`
    steps; falls back to the flat film when the residual misbehaves.
    Returns (used_warm, steps_taken).  Inputs, prediction, the predicted state
    and the residual statistics are all computed on the device."""
    x, _ = features_dev(sim, wl)
    d = net.predict_dev(x, (wl.nz, wl.ny, wl.nx))
    sim.warm_apply(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, d)
    sim.step(1)
    sim.field_check()  # keeps the densities after the first step
    sim.step(window)
    c1 = sim.field_check()
    sim.step(window)
    c2 = sim.field_check()
    # finite, no negative density, velocities below the low-Mach limit, and a
    # density change that decays from the first window to the second
    ok = all(c[0] == 1.0 and c[1] >= 0.0 and c[2] <= u_limit for c in (c1, c2)) and c2[3] <= grow * c1[3]
    if ok:
        return True, 2 * window + 1
    sim.set_film(wl.h_top, I.RHO_MAJ, I.RHO_MIN, I.RHO_MIX, wl.jitter())
    return False, 2 * window + 1


def force_traces(sims, total, every):
    """Capsule force z-component of every simulation every `every` steps
    (one batch); returns [len(sims)][total // every]."""
    batch = cfm.Batch(sims)
    out = []
    for _ in range(total // every):
        batch.step(every)
        out.append([s.capsule_force(0)[0][2] for s in sims])
    batch.close()
    return np.array(out).T


def settle_step(trace, every, f_eq, tol=0.01):
    """First sample step after which the trace stays within tol of f_eq
    (None when it never does)."""
    ok = np.abs(trace - f_eq) <= tol * abs(f_eq)
    for k in range(len(ok)):
        if ok[k:].all():
            return (k + 1) * every
    return None


def convergence(net, wls, total=8000, every=50, tol=0.01):
    """Flat-film and warm-started runs of the set-ups wls: steps until the
    capsule force settles within tol of its equilibrium (the mean of the last
    five samples of the flat-film run), and the warm starts that fell back.
    Also the wall time of one warm start (inference, predicted state, judging
    steps) and of one lattice step within the batch of force traces."""
    import time
    plain = [cfm.Simulation.from_workload(w) for w in wls]
    warmed, used = [], []
    t_warm = 0.0
    for w in wls:
        s = cfm.Simulation.from_workload(w)
        t0 = time.perf_counter()
        u, _ = warm_start(s, w, net)
        s.sync()
        t_warm += time.perf_counter() - t0
        warmed.append(s)
        used.append(u)
    t0 = time.perf_counter()
    fp = force_traces(plain, total, every)
    t_plain = time.perf_counter() - t0
    fw = force_traces(warmed, total, every)
    res = []
    for k in range(len(wls)):
        f_eq = fp[k, -5:].mean()
        res.append((settle_step(fp[k], every, f_eq, tol), settle_step(fw[k], every, f_eq, tol), used[k]))
    for s in plain + warmed:
        s.close()
    timing = dict(warm_start_seconds=t_warm / len(wls), step_seconds=t_plain / (total * len(wls)))
    return res, timing


# ----------------------------------------------------------- the U-net path
# The 3-D U-net (unet.py) trained on the sweep's generator: capsule pairs at
# distances 2.2R..6R with moduli 1e-3..1e-1 or rigid and films 0.2R..0.6R.
# Its density head gives the warm start of the coupled run (set up and judged
# as above); its displacement head the deformation of free capsules.

def pair_dataset(wls_fixed, wls_free, eq_steps, def_steps, chunk=64):
    """Training data of the U-net generated by the method.  Per set-up: the
    network inputs [4][V], density targets [2][V] and fluid mask [V] of the
    fixed-capsule run after eq_steps; the capsules' reference node positions
    [nodes][3] (lattice units) and their deformation after def_steps of the
    free run (each node's displacement minus its capsule's mean displacement)
    [nodes][3].  The runs go in batches of `chunk` lattices, each freed once
    its data is read."""
    X, T, M = [], [], []
    for i0 in range(0, len(wls_fixed), chunk):
        part = wls_fixed[i0:i0 + chunk]
        for s, w in zip(equilibrate(part, eq_steps), part):
            x, mask = features(s, w)
            X.append(x.reshape(N_IN, -1))
            T.append(target_of(s, w).reshape(N_OUT, -1))
            M.append(mask.reshape(-1))
            s.close()
    Xn, D = [], []
    for i0 in range(0, len(wls_free), chunk):
        part = wls_free[i0:i0 + chunk]
        for s, w in zip(equilibrate(part, def_steps), part):
            ref, dis = [], []
            for k, cap in enumerate(w.capsules):
                X0, _ = cap.mesh()
                X1 = s.capsule_state(k)["X"]
                ref.append(X0)
                dis.append((X1 - X1.mean(0)) - (X0 - X0.mean(0)))
            Xn.append(np.concatenate(ref))
            D.append(np.concatenate(dis))
            s.close()
    f32 = lambda a: np.ascontiguousarray(np.stack(a), np.float32)  # noqa: E731
    return dict(X=f32(X), T=f32(T), M=f32(M), Xn=f32(Xn), D=f32(D),
                shape=(wls_fixed[0].nz, wls_fixed[0].ny, wls_fixed[0].nx))


def train_unet(net, data, steps, batch=4, lr=1e-3, wx=1.0, seed=0, log=None):
    """Adam on mini-batches of the U-net data; returns the losses."""
    torch = net.torch
    from . import unet as U
    rng = np.random.default_rng(seed)
    nz, ny, nx = data["shape"]
    V = nz * ny * nx
    n, nodes = data["X"].shape[0], data["Xn"].shape[1]
    dev = net.dev
    losses = []
    for it in range(steps):
        idx = np.sort(rng.choice(n, size=min(batch, n), replace=False))
        b = len(idx)
        xf = torch.from_numpy(data["X"][idx]).to(dev)
        x = torch.empty(b * V * U.CIN, dtype=torch.bfloat16, device=dev)
        for k in range(b):
            cfm._check(cfm._lib.cf_unet_pack(_p(xf[k]), U.N_FEAT, V, U.CIN, _p(x[k * V * U.CIN:]),
                                             C.c_void_p(net.stream)))
        t = torch.from_numpy(data["T"][idx]).to(dev)
        m = torch.from_numpy(data["M"][idx]).to(dev)
        Xn = torch.from_numpy(data["Xn"][idx]).to(dev)
        D = torch.from_numpy(data["D"][idx]).to(dev)
        loss = net.train_step(x, (b, nz, ny, nx), t, m, float(data["M"][idx].sum()), Xn, D, nodes, lr=lr,
                              wd=1.0, wx=wx)
        losses.append(loss)
        if log and it % 50 == 0:
            log(f"step {it}: loss {loss:.4e}")
    return losses


def sample_field(field, X):
    """Trilinear samples of a vector field [3][nz][ny][nx] at positions X
    [k][3] (lattice units, clamped into the grid) -> [k][3] (host)."""
    c, nz, ny, nx = field.shape
    p = np.clip(X, 0, [nx - 1.001, ny - 1.001, nz - 1.001])
    i0 = np.floor(p).astype(int)
    f = p - i0
    out = np.zeros((X.shape[0], c))
    for k in range(8):
        dx, dy, dz = k & 1, (k >> 1) & 1, k >> 2
        wgt = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
        out += wgt[:, None] * field[:, i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx].T
    return out


def lateral_traces(sims, total, every):
    """Lateral force between capsules 0 and 1 of every simulation every
    `every` steps (one batch); returns ([len(sims)][total // every], seconds
    per lattice step)."""
    import time
    batch = cfm.Batch(sims)
    out = []
    t0 = time.perf_counter()
    for _ in range(total // every):
        batch.step(every)
        out.append(batch.lateral_forces(0, 1))
    dt = time.perf_counter() - t0
    batch.close()
    return np.array(out).T, dt / (total * len(sims))


def time_to_force(model_path, wls, total, every, tol=0.01):
    """Plain (flat film) and warm-started runs of the pair set-ups wls in
    batches: the steps after which the lateral force stays within tol of its
    converged value (the mean of the plain run's last five samples), whether
    each warm start was kept, and the wall times (one warm start; one
    lattice step within the batch).  The warm start runs inside the library
    (cf_warmstart) on the network saved at model_path (UNet.save)."""
    import time
    plain = [cfm.Simulation.from_workload(w) for w in wls]
    warmed, used = [], []
    t_warm = 0.0
    model = cfm.Model(model_path)
    for w in wls:
        s = cfm.Simulation.from_workload(w)
        t0 = time.perf_counter()
        u, _ = s.warmstart(model, w.h_top, w.capsules[0].kS, jitter=w.jitter())
        t_warm += time.perf_counter() - t0
        warmed.append(s)
        used.append(u)
    model.close()
    fp, step_plain = lateral_traces(plain, total, every)
    fw, step_warm = lateral_traces(warmed, total, every)
    res = []
    for k in range(len(wls)):
        f_eq = fp[k, -5:].mean()
        res.append(dict(plain=settle_step(fp[k], every, f_eq, tol), warm=settle_step(fw[k], every, f_eq, tol),
                        kept=bool(used[k]), f_eq=float(f_eq), f_warm_end=float(fw[k, -1])))
    for s in plain + warmed:
        s.close()
    return res, dict(warm_start_seconds=t_warm / len(wls), step_seconds=step_plain, step_seconds_warm=step_warm)
