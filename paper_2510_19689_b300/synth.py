"""Seeded synthetic inputs for TabNet inference: model parameters, the weight
blob that ``tabnet_create`` reads, and feature rows.

This module draws random numbers and serialises them.  It holds none of the
TabNet arithmetic (no BN, no GLU, no sparsemax): both the CUDA path (through
the blob) and the FP64 oracle (through the parameter dict) consume what it
produces, so the two sides see bit-identical weights and rows.

Workloads.  The paper evaluates TabNet (n_d = n_a = 8, three decision steps,
Sec. IV-A) on HR, census and labour tables that are not available here; the
three model shapes below stand in for them with seeded data of the same
width and value mix:

* ``c1``  14 inputs (6 numeric N(0,1), 8 categorical with cardinalities
  2..42, embedding dim 1), n_d = n_a = 8, 3 steps, gamma 1.3, 2 classes.
* ``c2``  35 inputs (13 lognormal(0,1) + 13 ordinal integers 1..5 stored as
  float, 9 categorical with cardinalities 2..10, embedding dim 1),
  n_d = n_a = 32, 5 steps, gamma 1.5, 2 classes.
* ``c3``  100 inputs (40 N(0,1) + 40 lognormal(0,1), each entry exactly 0
  with probability 0.05; 20 categorical with cardinalities 2..1000,
  embedding dim 4), n_d = n_a = 64, 10 steps, gamma 1.3, 3 classes.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the
i-th output of a stream with state s is mix(s + i * 0x9E3779B97F4A7C15).
Uniforms take the top 53 bits; normals use Box-Muller.
"""
from __future__ import annotations

import dataclasses
import math
import struct
from typing import Dict, List, Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class SplitMix64:
    """Sequential SplitMix64 stream, vectorised over blocks of draws."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + idx * _GOLDEN
            self.state = np.uint64(self.state + np.uint64(n) * _GOLDEN)
        return _mix64(z)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_range(self, n: int, lo: float, hi: float) -> np.ndarray:
        return lo + (hi - lo) * self.uniform(n)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (cosine branch)."""
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, n: int, hi: int) -> np.ndarray:
        """n integers uniform on [0, hi) (floor of a scaled uniform)."""
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)


# --------------------------------------------------------------------------
# Model specification
# --------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class TabNetSpec:
    n_num: int
    cat_card: tuple
    cat_emb_dim: tuple
    n_d: int
    n_a: int
    n_steps: int
    gamma: float
    n_classes: int
    n_shared: int = 2
    n_indep: int = 2
    bn_eps: float = 1e-5

    @property
    def n_cat(self) -> int:
        return len(self.cat_card)

    @property
    def d_emb(self) -> int:
        """Width D_e after the embedding lookup (numeric + embedded columns)."""
        return self.n_num + int(sum(self.cat_emb_dim))

    @property
    def n_feat(self) -> int:
        return self.n_num + self.n_cat

    @property
    def n_hidden(self) -> int:
        return self.n_d + self.n_a


def _c1_cards() -> tuple:
    return tuple(2 + int(round(40 * j / 7)) for j in range(8))


def _c3_cards() -> tuple:
    return tuple(int(round(2 * 500 ** (j / 19))) for j in range(20))


SPECS: Dict[str, TabNetSpec] = {
    "c1": TabNetSpec(n_num=6, cat_card=_c1_cards(), cat_emb_dim=(1,) * 8,
                     n_d=8, n_a=8, n_steps=3, gamma=1.3, n_classes=2),
    "c2": TabNetSpec(n_num=26, cat_card=tuple(2 + j for j in range(9)),
                     cat_emb_dim=(1,) * 9, n_d=32, n_a=32, n_steps=5,
                     gamma=1.5, n_classes=2),
    "c3": TabNetSpec(n_num=80, cat_card=_c3_cards(), cat_emb_dim=(4,) * 20,
                     n_d=64, n_a=64, n_steps=10, gamma=1.3, n_classes=3),
}

#: rows of the throughput workload for each model shape
ROWS = {"c1": 1024, "c2": 65536, "c3": 1048576}
#: config number used in the seeds (weights 1000 + k, data 2000 + k)
CONFIG_NUMBER = {"c1": 1, "c2": 2, "c3": 3}


def weight_seed(name: str) -> int:
    return 1000 + CONFIG_NUMBER[name]


def data_seed(name: str) -> int:
    return 2000 + CONFIG_NUMBER[name]


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------

def _he_uniform(rng: SplitMix64, rows: int, fan_in: int) -> np.ndarray:
    bound = math.sqrt(6.0 / fan_in)
    return rng.uniform_range(rows * fan_in, -bound, bound).reshape(rows, fan_in)


def _bn(rng: SplitMix64, n: int, affine: str) -> Dict[str, np.ndarray]:
    mean = 0.1 * rng.normal(n)
    var = rng.uniform_range(n, 0.5, 2.0)
    if affine == "identity":
        weight = np.ones(n)
        bias = np.zeros(n)
    elif affine == "random":
        weight = rng.uniform_range(n, 0.5, 1.5)
        bias = 0.1 * rng.normal(n)
    else:
        raise ValueError(affine)
    return {k: v.astype(np.float32) for k, v in
            dict(mean=mean, var=var, weight=weight, bias=bias).items()}


def make_params(spec: TabNetSpec, seed: int, bn_affine: str = "identity") -> dict:
    """Seeded parameters of one TabNet model (all float32 arrays).

    FC weights are He-uniform U(+-sqrt(6/fan_in)); embedding tables N(0,1);
    BN running means N(0, 0.1^2), variances U(0.5, 2); BN affine weight/bias
    are 1/0 (``identity``) or U(0.5,1.5)/N(0,0.1^2) (``random``); the final
    bias is U(+-1/sqrt(n_d)).
    """
    rng = SplitMix64(seed)
    N = spec.n_hidden
    De = spec.d_emb
    p: dict = dict(
        n_num=spec.n_num, cat_card=list(spec.cat_card),
        cat_emb_dim=list(spec.cat_emb_dim), n_d=spec.n_d, n_a=spec.n_a,
        n_steps=spec.n_steps, n_shared=spec.n_shared, n_indep=spec.n_indep,
        n_classes=spec.n_classes, gamma=float(spec.gamma),
        bn_eps=float(spec.bn_eps),
    )
    p["emb"] = [rng.normal(c * e).reshape(c, e).astype(np.float32)
                for c, e in zip(spec.cat_card, spec.cat_emb_dim)]
    p["bn0"] = _bn(rng, De, bn_affine)
    p["shared_fc"] = [
        _he_uniform(rng, 2 * N, De if l == 0 else N).astype(np.float32)
        for l in range(spec.n_shared)]
    ft = []
    for s in range(spec.n_steps + 1):
        shared_bn = [_bn(rng, 2 * N, bn_affine) for _ in range(spec.n_shared)]
        indep_fc, indep_bn = [], []
        for l in range(spec.n_indep):
            k = De if (spec.n_shared == 0 and l == 0) else N
            indep_fc.append(_he_uniform(rng, 2 * N, k).astype(np.float32))
            indep_bn.append(_bn(rng, 2 * N, bn_affine))
        ft.append(dict(shared_bn=shared_bn, indep_fc=indep_fc, indep_bn=indep_bn))
    p["ft"] = ft
    p["att"] = [dict(fc=_he_uniform(rng, De, spec.n_a).astype(np.float32),
                     bn=_bn(rng, De, bn_affine))
                for _ in range(spec.n_steps)]
    p["final_w"] = _he_uniform(rng, spec.n_classes, spec.n_d).astype(np.float32)
    bound = 1.0 / math.sqrt(spec.n_d)
    p["final_b"] = rng.uniform_range(spec.n_classes, -bound, bound).astype(np.float32)
    return p


def spec_of(params: dict) -> TabNetSpec:
    return TabNetSpec(
        n_num=params["n_num"], cat_card=tuple(params["cat_card"]),
        cat_emb_dim=tuple(params["cat_emb_dim"]), n_d=params["n_d"],
        n_a=params["n_a"], n_steps=params["n_steps"], gamma=params["gamma"],
        n_classes=params["n_classes"], n_shared=params["n_shared"],
        n_indep=params["n_indep"], bn_eps=params["bn_eps"])


# --------------------------------------------------------------------------
# Feature rows
# --------------------------------------------------------------------------

def make_rows(name: str, rows: int, seed: Optional[int] = None,
              spec: Optional[TabNetSpec] = None):
    """Seeded feature rows for workload ``name`` (x_num float32 [rows, n_num],
    x_cat int32 [rows, n_cat]).  ``spec`` overrides the model shape for
    ``name == "generic"`` (numeric N(0,1), categorical uniform)."""
    if seed is None:
        seed = data_seed(name)
    rng = SplitMix64(seed)
    spec = SPECS[name] if spec is None else spec
    if name == "c2":
        logn = np.exp(rng.normal(rows * 13)).reshape(rows, 13)
        ordinal = (1 + rng.integers(rows * 13, 5)).reshape(rows, 13)
        x_num = np.concatenate([logn, ordinal.astype(np.float64)], axis=1)
    elif name == "c3":
        nrm = rng.normal(rows * 40).reshape(rows, 40)
        logn = np.exp(rng.normal(rows * 40)).reshape(rows, 40)
        x_num = np.concatenate([nrm, logn], axis=1)
        zero = rng.uniform(rows * 80).reshape(rows, 80) < 0.05
        x_num[zero] = 0.0
    else:
        x_num = rng.normal(rows * spec.n_num).reshape(rows, spec.n_num)
    x_cat = np.zeros((rows, spec.n_cat), dtype=np.int32)
    for j, card in enumerate(spec.cat_card):
        x_cat[:, j] = rng.integers(rows, card).astype(np.int32)
    return np.ascontiguousarray(x_num, dtype=np.float32), x_cat


def segment_rows(n_segments: int, max_rows: int, seed: int) -> np.ndarray:
    """Row counts of uneven request batches: floor(exp(U(0, ln(max+1))))
    clamped to [1, max] (log-uniform sizes)."""
    rng = SplitMix64(seed)
    u = rng.uniform(n_segments)
    r = np.floor(np.exp(u * math.log(max_rows + 1))).astype(np.int64)
    return np.clip(r, 1, max_rows)


# --------------------------------------------------------------------------
# Weight blob (format version 1)
# --------------------------------------------------------------------------
#
# Header, 96 bytes, little-endian:
#   u32 magic 0x4E424154 ("TABN"), u32 version 1, u32 header_bytes 96,
#   u32 flags 0, u64 payload_bytes, u64 payload_hash,
#   i32 n_num, n_cat, n_d, n_a, n_steps, n_shared, n_indep, n_classes,
#   f64 gamma, f64 bn_eps, 16 reserved bytes (zero).
# Payload, in this order (i32 then float32, C order):
#   cat_card[n_cat], cat_emb_dim[n_cat],
#   emb_j [card_j, emb_dim_j] for each categorical j,
#   bn0 {mean, var, weight, bias} [D_e] each,
#   shared_fc_l [2N, K_l] for l < n_shared (K_0 = D_e, else N),
#   for each feature transformer s = 0..n_steps:
#       shared_bn_l {mean, var, weight, bias} [2N] for l < n_shared,
#       for l < n_indep: indep_fc [2N, K] then indep_bn {..} [2N],
#   for each step i = 1..n_steps: att_fc [D_e, n_a] then att_bn {..} [D_e],
#   final_w [C, n_d], final_b [C].
# payload_hash = sum over little-endian u32 words w_i of
#   mix64(w_i XOR (i+1) * 0x9E3779B97F4A7C15)  (mod 2^64).

BLOB_MAGIC = 0x4E424154
BLOB_VERSION = 1
HEADER_BYTES = 96


def payload_hash(payload: bytes) -> int:
    assert len(payload) % 4 == 0
    w = np.frombuffer(payload, dtype="<u4").astype(np.uint64)
    idx = np.arange(1, w.size + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _mix64(w ^ (idx * _GOLDEN))
        return int(np.sum(h, dtype=np.uint64))


def _bn_bytes(bn) -> List[bytes]:
    return [np.ascontiguousarray(bn[k], dtype="<f4").tobytes()
            for k in ("mean", "var", "weight", "bias")]


def to_blob(params: dict) -> bytes:
    parts: List[bytes] = []
    f4 = lambda a: np.ascontiguousarray(a, dtype="<f4").tobytes()
    parts.append(np.asarray(params["cat_card"], dtype="<i4").tobytes())
    parts.append(np.asarray(params["cat_emb_dim"], dtype="<i4").tobytes())
    for t in params["emb"]:
        parts.append(f4(t))
    parts += _bn_bytes(params["bn0"])
    for w in params["shared_fc"]:
        parts.append(f4(w))
    for ft in params["ft"]:
        for bn in ft["shared_bn"]:
            parts += _bn_bytes(bn)
        for w, bn in zip(ft["indep_fc"], ft["indep_bn"]):
            parts.append(f4(w))
            parts += _bn_bytes(bn)
    for att in params["att"]:
        parts.append(f4(att["fc"]))
        parts += _bn_bytes(att["bn"])
    parts.append(f4(params["final_w"]))
    parts.append(f4(params["final_b"]))
    payload = b"".join(parts)
    header = struct.pack(
        "<IIIIQQ8idd16x", BLOB_MAGIC, BLOB_VERSION, HEADER_BYTES, 0,
        len(payload), payload_hash(payload),
        params["n_num"], len(params["cat_card"]), params["n_d"], params["n_a"],
        params["n_steps"], params["n_shared"], params["n_indep"],
        params["n_classes"], float(params["gamma"]), float(params["bn_eps"]))
    assert len(header) == HEADER_BYTES
    return header + payload


def load_config(name: str, rows: Optional[int] = None, bn_affine: str = "identity"):
    """(params, blob, x_num, x_cat) for workload ``name`` at its seeds."""
    spec = SPECS[name]
    params = make_params(spec, weight_seed(name), bn_affine)
    x_num, x_cat = make_rows(name, ROWS[name] if rows is None else rows)
    return params, to_blob(params), x_num, x_cat
