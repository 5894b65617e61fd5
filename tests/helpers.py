"""Shared test helpers: building/loading the library, packing, and oracle adapters."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def ensure_built():
    """Builds libnqs.so if needed; build.py is loaded by path, since importing the package
    needs the library."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_nqs_build", os.path.join(ROOT, "paper_2601_20782_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def nqs():
    ensure_built()
    import paper_2601_20782_b300 as pkg
    return pkg


def pack_np(s):
    """[n, N] +-1 -> [n, W] uint32 packed words (numpy)."""
    s = np.asarray(s)
    n, N = s.shape
    W = (N + 31) // 32
    bits = np.zeros((n, W * 32), dtype=np.uint64)
    bits[:, :N] = s > 0
    words = (bits.reshape(n, W, 32) << np.arange(32, dtype=np.uint64)).sum(axis=2)
    return words.astype(np.uint32)


def unpack_np(words, N):
    w = np.asarray(words).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return (bits.reshape(w.shape[0], -1)[:, :N].astype(np.int8) * 2 - 1).astype(np.int8)


def unpack_accept_bits(bits, N):
    """[C, T, W] words -> [C, T, N] bool."""
    C, T, W = bits.shape
    w = np.asarray(bits).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    b = (w[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return b.reshape(C, T, W * 32)[:, :, :N].astype(bool)


def to_words_tensor(words_np, device="cuda"):
    import torch
    return torch.from_numpy(np.asarray(words_np, dtype=np.uint32).view(np.int32).copy()).to(device)


def words_from_tensor(t):
    return t.cpu().numpy().view(np.uint32)
