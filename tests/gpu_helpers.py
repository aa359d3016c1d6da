"""Shared helpers of the GPU parity tests (oracle values vs the C-ABI)."""
import numpy as np
import torch

from oracle import ctmrg as C

KEYS = ("C1", "T1k", "T1b", "C2", "T2k", "T2b", "C3", "T3b", "T3k", "C4", "T4b", "T4k")


FIRST = ("T1k", "T2k", "T3b", "T4b")   # [chi_E, D, chi_I]; the others [chi_I, D, chi_E]


def pad_env(e, chi, chi_I=None):
    """oracle site environment (grown dims) -> zero-padded to chi_E = chi and chi_I"""
    ci = chi_I or chi
    out = {}
    for k in KEYS:
        t = e[k].detach()
        if t.dim() == 2:
            z = torch.zeros(chi, chi, dtype=torch.float64)
            z[:t.shape[0], :t.shape[1]] = t
        else:
            a, b = (chi, ci) if k in FIRST else (ci, chi)
            z = torch.zeros(a, t.shape[1], b, dtype=torch.float64)
            z[:t.shape[0], :, :t.shape[2]] = t
        out[k] = z
    return out


def env_max_rel_diff(S, env_oracle, chi, chi_I=None):
    """max over sites/keys of |gpu - oracle| / max|oracle|"""
    Lx, Ly = len(env_oracle), len(env_oracle[0])
    worst = 0.0
    for x in range(Lx):
        for y in range(Ly):
            g = S.env(x, y)
            o = pad_env(env_oracle[x][y], chi, chi_I)
            for k in KEYS:
                d = (g[k].cpu() - o[k]).abs().max().item() / max(o[k].abs().max().item(), 1e-300)
                worst = max(worst, d)
    return worst
