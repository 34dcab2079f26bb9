"""Shared test utilities: parity metrics between the CUDA path and the oracle."""
import numpy as np


def q_rel_err(Qg, Qo):
    """Per-component error max_ij |Qg - Qo| / max(max_ij |Qo_c|, max_ij rho_o): the macro-field
    parity metric (the density floor handles components that are identically ~0)."""
    Qg = np.asarray(Qg).reshape(6, -1)
    Qo = np.asarray(Qo).reshape(6, -1)
    rho_max = np.max(np.abs(Qo[0]))
    return np.array([np.max(np.abs(Qg[c] - Qo[c])) / max(np.max(np.abs(Qo[c])), rho_max)
                     for c in range(6)])


def rel_max(a, b, floor=1e-300):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor)


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
