"""Plain FP32 unfused TabNet forward on the GPU with PyTorch eager ops.

This is the comparison point the fused kernels are measured against (the
straightforward way to run the deployed TabNet of Sec. IV-A on a GPU: one
library call per operation, every intermediate in HBM).  TF32 is disabled
so that every FC is an FP32 GEMM; sparsemax is the sort-and-threshold rule.
It shares no code with the fused kernels or with the FP64 oracle.
"""
from __future__ import annotations

import math

import numpy as np
import torch


class UnfusedTabNet:
    def __init__(self, params: dict, device="cuda"):
        torch.backends.cuda.matmul.allow_tf32 = False
        torch.backends.cudnn.allow_tf32 = False
        dev = torch.device(device)
        f32 = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float32), device=dev)
        eps = params["bn_eps"]
        self.n_d = params["n_d"]
        self.n_steps = params["n_steps"]
        self.gamma = float(params["gamma"])
        self.n_num = params["n_num"]

        def bn(b):  # inference BN as (scale, shift)
            s = f32(b["weight"]) / torch.sqrt(f32(b["var"]) + eps)
            return s, f32(b["bias"]) - f32(b["mean"]) * s

        self.emb = [f32(t) for t in params["emb"]]
        self.bn0 = bn(params["bn0"])
        shared = [f32(w) for w in params["shared_fc"]]
        self.ft = []
        for ftp in params["ft"]:
            layers = [(w, bn(b)) for w, b in zip(shared, ftp["shared_bn"])]
            layers += [(f32(w), bn(b)) for w, b in zip(ftp["indep_fc"], ftp["indep_bn"])]
            self.ft.append(layers)
        self.att = [(f32(a["fc"]), bn(a["bn"])) for a in params["att"]]
        self.wf = f32(params["final_w"])
        self.bf = f32(params["final_b"])
        groups = [1] * params["n_num"] + list(params["cat_emb_dim"])
        self.group_index = torch.as_tensor(np.repeat(np.arange(len(groups)), groups), device=dev)
        self.n_feat = len(groups)

    @staticmethod
    def sparsemax(z):
        zs, _ = torch.sort(z, dim=-1, descending=True)
        cs = zs.cumsum(-1)
        k = torch.arange(1, z.shape[-1] + 1, device=z.device, dtype=z.dtype)
        ok = 1 + k * zs > cs
        kstar = ok.sum(-1, keepdim=True)
        tau = (cs.gather(-1, kstar - 1) - 1) / kstar.to(z.dtype)
        return torch.clamp(z - tau, min=0)

    def _ft(self, s, x):
        for l, (w, (sc, sh)) in enumerate(self.ft[s]):
            u = torch.nn.functional.linear(x, w) * sc + sh
            n = u.shape[-1] // 2
            g = u[:, :n] * torch.sigmoid(u[:, n:])
            x = g if l == 0 else (x + g) * math.sqrt(0.5)
        return x

    @torch.no_grad()
    def forward(self, x_num, x_cat):
        cols = [x_num] + [t[x_cat[:, j].long()] for j, t in enumerate(self.emb)]
        f = torch.cat(cols, dim=1) * self.bn0[0] + self.bn0[1]
        o = self._ft(0, f)
        a = o[:, self.n_d:]
        prior = torch.ones_like(f)
        acc = torch.zeros((f.shape[0], self.n_d), device=f.device)
        agg = torch.zeros_like(f)
        masks = []
        for i in range(self.n_steps):
            w, (sc, sh) = self.att[i]
            z = (torch.nn.functional.linear(a, w) * sc + sh) * prior
            m = self.sparsemax(z)
            prior = prior * (self.gamma - m)
            o = self._ft(i + 1, m * f)
            d = torch.relu(o[:, :self.n_d])
            a = o[:, self.n_d:]
            acc = acc + d
            agg = agg + d.sum(1, keepdim=True) * m
            masks.append(m)
        logits = torch.nn.functional.linear(acc, self.wf) + self.bf
        agg_d = torch.zeros((f.shape[0], self.n_feat), device=f.device).index_add_(1, self.group_index, agg)
        tot = agg_d.sum(1, keepdim=True)
        agg_d = torch.where(tot > 0, agg_d / torch.where(tot > 0, tot, torch.ones_like(tot)), torch.zeros_like(agg_d))
        return logits, torch.stack(masks, 1), agg_d
