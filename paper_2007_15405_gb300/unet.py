"""3-D U-net of the learned warm start, on the library's tensor-core layers.

Every layer, gradient, loss and optimiser step runs in the CUDA library
(cf_unet_conv_tc on the tcgen05 tensor cores, or cf_unet_conv on mma.sync /
cf_unet_flip / cf_unet_wgrad / cf_unet_relu_grad /
cf_unet_pool / cf_unet_upsample / cf_unet_concat / cf_unet_split /
cf_unet_loss / cf_adam: bfloat16 activations and weights, fp32 accumulation
on the tensor cores, fp32 gradients and master weights, sums in fixed order);
this module holds the device buffers (torch tensors) and orders the calls.

Architecture (channels-last, widths w0, w1, w2 = 32, 64, 128 by default):

    x (16: four set-up features, zero-padded)
    e0 = conv(16->w0), conv(w0->w0)                       full grid
    e1 = conv(w0->w1), conv(w1->w1) of pool(e0)           1/2
    m  = conv(w1->w2), conv(w2->w2) of pool(e1)           1/4
    d1 = conv(w1+w2->w1), conv(w1->w1) of [e1, up(m)]     1/2
    d0 = conv(w0+w1->w0), conv(w0->w0) of [e0, up(d1)]    full
    head = conv(w0->16) of d0, no activation: channels 0, 1 the density
           corrections, 2..4 a displacement field (lattice units)

3x3x3 convolutions with zero padding and ReLU, 2x2x2 average pooling,
nearest-neighbour upsampling; lattice dimensions must be multiples of 4.
With the default widths the network has 1.43 million parameters.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import capfilm as cfm

CIN = 16     # input channels (features padded)
HEAD = 16    # output channels (5 used)
N_FEAT = 4   # set-up features per node (cf_warm_features)
WCHUNKS = 16  # voxel chunks of the weight gradient


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class UNet:
    def __init__(self, widths=(32, 64, 128), seed=0, device="cuda", tensor_memory=True):
        import torch
        self.torch = torch
        self.dev = device
        self.tensor_memory = tensor_memory  # tcgen05 convolutions (else mma.sync)
        w0, w1, w2 = widths
        self.widths = widths
        self.specs = [("e0a", CIN, w0, True), ("e0b", w0, w0, True), ("e1a", w0, w1, True),
                      ("e1b", w1, w1, True), ("ma", w1, w2, True), ("mb", w2, w2, True),
                      ("d1a", w1 + w2, w1, True), ("d1b", w1, w1, True), ("d0a", w0 + w1, w0, True),
                      ("d0b", w0, w0, True), ("head", w0, HEAD, False)]
        rng = np.random.default_rng(seed)
        self.w, self.wb, self.b = {}, {}, {}
        self.mw, self.vw, self.mb, self.vb = {}, {}, {}, {}
        for name, ci, co, relu in self.specs:
            std = math.sqrt(2.0 / (27 * ci)) if relu else 0.1 * math.sqrt(1.0 / (27 * ci))
            w = (rng.standard_normal((27, co, ci)) * std).astype(np.float32)
            self.w[name] = torch.from_numpy(w).to(device).reshape(-1)
            self.wb[name] = torch.empty(w.size, dtype=torch.bfloat16, device=device)
            self.b[name] = torch.zeros(co, dtype=torch.float32, device=device)
            self.mw[name] = torch.zeros_like(self.w[name])
            self.vw[name] = torch.zeros_like(self.w[name])
            self.mb[name] = torch.zeros_like(self.b[name])
            self.vb[name] = torch.zeros_like(self.b[name])
        self.stream = torch.cuda.current_stream().cuda_stream
        self._to_bf16()
        self.t = 0
        big = max(ci * co for _, ci, co, _ in self.specs)
        self.part = torch.empty(WCHUNKS * 27 * big, dtype=torch.float32, device=device)

    @property
    def n_params(self):
        return sum(self.w[k].numel() + self.b[k].numel() for k in self.w)

    def _s(self):
        return C.c_void_p(self.stream)

    def _to_bf16(self):
        L = cfm.load_library()
        for k in self.w:
            cfm._check(L.cf_to_bf16(_p(self.w[k]), _p(self.wb[k]), self.w[k].numel(), self._s()))

    def _spec(self, name):
        return next(s for s in self.specs if s[0] == name)

    # ------------------------------------------------------------- forward
    def _conv_call(self, x, n, nz, ny, nx, ci, w, b, co, relu, out_f32, y):
        """One convolution: on the tcgen05 path (cf_unet_conv_tc) where the
        channel counts allow and self.tensor_memory is set, else mma.sync."""
        fn = cfm._lib.cf_unet_conv_tc if (self.tensor_memory and ci % 16 == 0 and co % 16 == 0
                                          and ci <= 256 and co <= 256) else cfm._lib.cf_unet_conv
        cfm._check(fn(_p(x), n, nz, ny, nx, ci, _p(w), _p(b), co, int(relu), int(out_f32), _p(y), self._s()))

    def _conv(self, name, x, grid, out_f32=False):
        torch = self.torch
        _, ci, co, relu = self._spec(name)
        n, nz, ny, nx = grid
        y = torch.empty(n * nz * ny * nx * co, device=self.dev,
                        dtype=torch.float32 if out_f32 else torch.bfloat16)
        self._conv_call(x, n, nz, ny, nx, ci, self.wb[name], self.b[name], co, relu, out_f32, y)
        return y

    def _pool(self, x, grid, c):
        torch = self.torch
        n, nz, ny, nx = grid
        y = torch.empty(x.numel() // 8, device=self.dev, dtype=torch.bfloat16)
        cfm._check(cfm._lib.cf_unet_pool(_p(x), n, nz, ny, nx, c, _p(y), self._s()))
        return y

    def _up(self, x, fine, c):
        torch = self.torch
        n, nz, ny, nx = fine
        y = torch.empty(x.numel() * 8, device=self.dev, dtype=torch.bfloat16)
        cfm._check(cfm._lib.cf_unet_upsample(_p(x), n, nz, ny, nx, c, _p(y), self._s()))
        return y

    def _cat(self, a, ca, b, cb, nv):
        torch = self.torch
        y = torch.empty(nv * (ca + cb), device=self.dev, dtype=torch.bfloat16)
        cfm._check(cfm._lib.cf_unet_concat(nv, _p(a), ca, _p(b), cb, _p(y), self._s()))
        return y

    def forward(self, x, grid):
        """x: bfloat16 [n][nz][ny][nx][16]; returns the activations (dict),
        'head' in float32 [n][nz][ny][nx][16]."""
        w0, w1, w2 = self.widths
        n, nz, ny, nx = grid
        g1 = (n, nz // 2, ny // 2, nx // 2)
        g2 = (n, nz // 4, ny // 4, nx // 4)
        a = {"x": x}
        a["e0a"] = self._conv("e0a", x, grid)
        a["e0b"] = self._conv("e0b", a["e0a"], grid)
        a["p1"] = self._pool(a["e0b"], grid, w0)
        a["e1a"] = self._conv("e1a", a["p1"], g1)
        a["e1b"] = self._conv("e1b", a["e1a"], g1)
        a["p2"] = self._pool(a["e1b"], g1, w1)
        a["ma"] = self._conv("ma", a["p2"], g2)
        a["mb"] = self._conv("mb", a["ma"], g2)
        a["u1"] = self._up(a["mb"], g1, w2)
        a["c1"] = self._cat(a["e1b"], w1, a["u1"], w2, int(np.prod(g1)))
        a["d1a"] = self._conv("d1a", a["c1"], g1)
        a["d1b"] = self._conv("d1b", a["d1a"], g1)
        a["u0"] = self._up(a["d1b"], grid, w1)
        a["c0"] = self._cat(a["e0b"], w0, a["u0"], w1, int(np.prod(grid)))
        a["d0a"] = self._conv("d0a", a["c0"], grid)
        a["d0b"] = self._conv("d0b", a["d0a"], grid)
        a["head"] = self._conv("head", a["d0b"], grid, out_f32=True)
        return a

    # ------------------------------------------------------------ backward
    def _layer_back(self, name, g, g2, act_in, act_out, grid, grads, need_gx=True):
        """Gradient g (float, + g2) of layer `name`'s output: adds the weight
        and bias gradients to grads and returns the input gradient (float)."""
        torch = self.torch
        L = cfm._lib
        _, ci, co, relu = self._spec(name)
        n, nz, ny, nx = grid
        m = n * nz * ny * nx * co
        gm = torch.empty(m, device=self.dev, dtype=torch.bfloat16)
        cfm._check(L.cf_unet_relu_grad(_p(g), _p(g2), _p(act_out) if relu else None, m, _p(gm), self._s()))
        gw, gb = grads[name]
        cfm._check(L.cf_unet_wgrad(_p(act_in), _p(gm), n, nz, ny, nx, ci, co, WCHUNKS, _p(self.part), _p(gw),
                                   _p(gb), self._s()))
        if not need_gx:
            return None
        wt = torch.empty_like(self.wb[name])
        cfm._check(L.cf_unet_flip(_p(self.wb[name]), ci, co, _p(wt), self._s()))
        gx = torch.empty(n * nz * ny * nx * ci, device=self.dev, dtype=torch.float32)
        self._conv_call(gm, n, nz, ny, nx, co, wt, None, ci, 0, 1, gx)
        return gx

    def backward(self, a, g_head, grid):
        """Weight and bias gradients (dict name -> (gw, gb), float) for the
        head gradient g_head (float, the shape of a['head'])."""
        torch = self.torch
        L = cfm._lib
        w0, w1, w2 = self.widths
        n, nz, ny, nx = grid
        g1 = (n, nz // 2, ny // 2, nx // 2)
        g2 = (n, nz // 4, ny // 4, nx // 4)
        nv0, nv1 = int(np.prod(grid)), int(np.prod(g1))
        grads = {k: (torch.zeros_like(self.w[k]), torch.zeros_like(self.b[k])) for k in self.w}
        f = lambda m: torch.empty(m, device=self.dev, dtype=torch.float32)  # noqa: E731
        s = self._s()
        g = self._layer_back("head", g_head, None, a["d0b"], None, grid, grads)
        g = self._layer_back("d0b", g, None, a["d0a"], a["d0b"], grid, grads)
        g = self._layer_back("d0a", g, None, a["c0"], a["d0a"], grid, grads)
        g_e0b_skip, g_u0 = f(nv0 * w0), f(nv0 * w1)
        cfm._check(L.cf_unet_split(nv0, _p(g), w0, w1, _p(g_e0b_skip), _p(g_u0), s))
        g = f(nv1 * w1)
        cfm._check(L.cf_unet_upsample_bwd(_p(g_u0), n, nz, ny, nx, w1, _p(g), s))
        g = self._layer_back("d1b", g, None, a["d1a"], a["d1b"], g1, grads)
        g = self._layer_back("d1a", g, None, a["c1"], a["d1a"], g1, grads)
        g_e1b_skip, g_u1 = f(nv1 * w1), f(nv1 * w2)
        cfm._check(L.cf_unet_split(nv1, _p(g), w1, w2, _p(g_e1b_skip), _p(g_u1), s))
        g = f(nv1 // 8 * w2)
        cfm._check(L.cf_unet_upsample_bwd(_p(g_u1), *g1, w2, _p(g), s))
        g = self._layer_back("mb", g, None, a["ma"], a["mb"], g2, grads)
        g = self._layer_back("ma", g, None, a["p2"], a["ma"], g2, grads)
        g_e1b_pool = f(nv1 * w1)
        cfm._check(L.cf_unet_pool_bwd(_p(g), *g1, w1, _p(g_e1b_pool), s))
        g = self._layer_back("e1b", g_e1b_skip, g_e1b_pool, a["e1a"], a["e1b"], g1, grads)
        g = self._layer_back("e1a", g, None, a["p1"], a["e1a"], g1, grads)
        g_e0b_pool = f(nv0 * w0)
        cfm._check(L.cf_unet_pool_bwd(_p(g), n, nz, ny, nx, w0, _p(g_e0b_pool), s))
        g = self._layer_back("e0b", g_e0b_skip, g_e0b_pool, a["e0a"], a["e0b"], grid, grads)
        self._layer_back("e0a", g, None, a["x"], a["e0a"], grid, grads, need_gx=False)
        return grads

    # ------------------------------------------------------------ training
    def loss_and_grad(self, a, grid, t, mask, msum, X=None, d=None, nodes=0, wd=1.0, wx=0.0):
        """(loss, head gradient) of the density corrections t [n][2][V]
        (mask [n][V], msum its sum) and, with nodes > 0, of the node
        displacements d at reference positions X (float [n][nodes][3])."""
        torch = self.torch
        n, nz, ny, nx = grid
        g = torch.empty_like(a["head"])
        loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        part = torch.empty(304 + n, dtype=torch.float64, device=self.dev)
        cfm._check(cfm._lib.cf_unet_loss(_p(a["head"]), n, nz, ny, nx, HEAD, _p(t), _p(mask), wd / msum,
                                         _p(X), _p(d), int(nodes), wx, _p(part), _p(g), _p(loss), self._s()))
        return loss, g

    def adam(self, grads, lr, b1=0.9, b2=0.999, eps=1e-8):
        L = cfm._lib
        self.t += 1
        for k in self.w:
            gw, gb = grads[k]
            cfm._check(L.cf_adam(_p(self.w[k]), _p(self.wb[k]), _p(gw), _p(self.mw[k]), _p(self.vw[k]),
                                 self.w[k].numel(), lr, b1, b2, eps, self.t, self._s()))
            cfm._check(L.cf_adam(_p(self.b[k]), None, _p(gb), _p(self.mb[k]), _p(self.vb[k]),
                                 self.b[k].numel(), lr, b1, b2, eps, self.t, self._s()))

    def train_step(self, x, grid, t, mask, msum, X=None, d=None, nodes=0, lr=1e-3, wd=1.0, wx=0.0):
        a = self.forward(x, grid)
        loss, g = self.loss_and_grad(a, grid, t, mask, msum, X, d, nodes, wd, wx)
        grads = self.backward(a, g, grid)
        self.adam(grads, lr)
        return float(loss.item())

    def save(self, path):
        """Weights file read by the library's cf_model_load: "CFUNET01", int32
        widths, then per layer int32 cin, cout, float32 weights [27][cout][cin]
        and biases [cout]."""
        import struct
        with open(path, "wb") as f:
            f.write(b"CFUNET01")
            f.write(struct.pack("<3i", *self.widths))
            for name, ci, co, _ in self.specs:
                f.write(struct.pack("<2i", ci, co))
                f.write(self.w[name].cpu().numpy().astype("<f4").tobytes())
                f.write(self.b[name].cpu().numpy().astype("<f4").tobytes())

    # ----------------------------------------------------------- inference
    def pack(self, feats, N):
        """Features float [4][N] (one lattice, device) -> bfloat16 [N][16]."""
        torch = self.torch
        x = torch.empty(N * CIN, device=self.dev, dtype=torch.bfloat16)
        cfm._check(cfm._lib.cf_unet_pack(_p(feats), N_FEAT, N, CIN, _p(x), self._s()))
        return x

    def predict_dev(self, feats, shape):
        """Density corrections float [2][N] (device) of one lattice of shape
        (nz, ny, nx) from its features float [4][N] (device)."""
        dens, _ = self.predict_both(feats, shape)
        return dens

    def predict_both(self, feats, shape):
        """(density corrections [2][N], displacement field [3][N]) float, device."""
        torch = self.torch
        nz, ny, nx = shape
        N = nz * ny * nx
        a = self.forward(self.pack(feats, N), (1, nz, ny, nx))
        dens = torch.empty(2 * N, device=self.dev, dtype=torch.float32)
        disp = torch.empty(3 * N, device=self.dev, dtype=torch.float32)
        cfm._check(cfm._lib.cf_unet_unpack(_p(a["head"]), 1, HEAD, N, 0, 2, _p(dens), self._s()))
        cfm._check(cfm._lib.cf_unet_unpack(_p(a["head"]), 1, HEAD, N, 2, 3, _p(disp), self._s()))
        torch.cuda.synchronize()  # the simulation reads the prediction on its own stream
        return dens, disp
