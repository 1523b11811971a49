"""Shared test helpers: golden-file readers and small seeded inputs."""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import torch

from paper_2503_06721_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table1():
    """rows of tests/golden/table1_representations.txt as dicts of Fractions."""
    rows = []
    with open(os.path.join(GOLDEN, "table1_representations.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rep, N, D, Tp, Tr, C2 = line.split()
            rows.append(dict(rep=rep, N=int(N), D=int(D), T_printed=Fraction(Tp),
                             T=Fraction(Tr), C2=Fraction(C2)))
    return rows


def gamma_blocks():
    """e_mu 2x2 blocks as printed in Sec. 2.2."""
    out = {}
    with open(os.path.join(GOLDEN, "gamma_basis.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            mu, *ent = line.split()
            vals = [complex(float(e.split(",")[0]), float(e.split(",")[1])) for e in ent]
            out[int(mu)] = np.array(vals).reshape(2, 2)
    return out


def su_n(count, N, seed, eps=1.0):
    """count random SU(N) matrices exp(i eps H) (numpy complex128)."""
    return synth.random_links(count, N, eps, seed).reshape(-1, N, N)[:count].numpy()


def spinor(nsites, D, seed, nrhs=1):
    return synth.gaussian_spinor(nsites, D, seed, nrhs=nrhs).numpy()


def hermitian(count, N, seed, stream=synth.STREAM_DIRECTION):
    return synth.gaussian_hermitian(count, N, seed, stream).numpy()


def links(dims, N, eps, seed, haar=False):
    V = int(np.prod(dims))
    U = synth.random_links(V, N, eps, seed)
    if haar:
        g = synth.haar_su_n(V, N, seed)
        U = synth.gauge_transform_links(U, g, dims)
    return U.numpy()


def unit_links(dims, N):
    V = int(np.prod(dims))
    return np.broadcast_to(np.eye(N, dtype=np.complex128), (V, 4, N, N)).copy()


def coords(dims):
    T, X, Y, Z = dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z),
                             indexing="ij")
    return np.stack([t, x, y, z], -1).reshape(-1, 4)


def rel_site_norm(a, b):
    """max_x |a(x) - b(x)|_2 / rms_x |b(x)|_2 over the leading (site) axis."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    d = np.sqrt((np.abs(a - b) ** 2).sum(1))
    rms = np.sqrt((np.abs(b) ** 2).sum(1).mean())
    return float(d.max() / rms) if rms > 0 else float(d.max())


def torch_expm(A):
    return torch.linalg.matrix_exp(torch.as_tensor(A)).numpy()
