"""Shared fixtures of the GPU tests: the built library, seeded inputs."""
import numpy as np
import torch

from paper_2206_14286_gb300 import build as B
from paper_2206_14286_gb300 import search as S

_built = False


def ensure_built():
    global _built
    if not _built:
        B.build()
        _built = True
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def db(X, metric, dtype, keep_f32=True):
    ensure_built()
    return S.Database(dev(X), metric=metric, dtype=dtype, keep_f32=keep_f32)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bf16_bits_to_f64(u8, rows, pitch, D):
    v = u8.view(torch.bfloat16).reshape(rows, pitch).float().cpu().numpy().astype(np.float64)
    return v[:, :D], v[:, D:]
