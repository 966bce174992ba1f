"""Shared set-up for the GPU parity tests: builds the library, makes seeded
inputs, and compares with the CPU oracle."""
from __future__ import annotations

import numpy as np

import hisq_inputs as hi

# Elementwise tolerances relative to the largest oracle magnitude, derived
# from the arithmetic: a stencil output sums 48 complex products, so the
# rounding bound is ~48 * u * max|term| with u = 2^-48 (double-float),
# 2^-53 (FP64) or 2^-24 (FP32), and a factor ~4 of slack.
TOL = {"f64": 1e-12, "f64_native": 1e-13, "mixed_f32": 2e-5,
       # 16-bit storage: each element rounded to 2^-11 (FP16) or 2^-8 (BF16)
       # relative, ~sqrt(48) growth over the 48 terms of a stencil output
       "mixed_f16": 1e-2, "mixed_bf16": 5e-2}


def torch_mod():
    import torch
    return torch


def ensure_built():
    from paper_1710_09745_gb300 import build
    build.build()


def make_solver(dims, mass, prec="f64", max_rhs=16, seed=1000, links=None, **kw):
    ensure_built()
    kw.setdefault("max_iter", 20000)
    from paper_1710_09745_gb300 import BlockCG
    if links is None:
        links = hi.random_links(dims, seed)
    fat, lng = links
    return BlockCG(dims, fat, lng, mass, prec=prec, max_rhs=max_rhs, **kw), fat, lng


def to_np(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
