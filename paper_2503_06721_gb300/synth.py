"""Seeded synthetic inputs: gauge links, gauge transformations and spinor fields.

This module holds no arithmetic of the Wilson-Dirac method itself.  It is the
one module that both the GPU library's tests/benchmark and the CPU oracle's
tests draw inputs from, so the two sides always see the same numbers.

Random numbers come from a counter-based generator written out from its
published definition: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), with Gaussian variates from the
Box-Muller transform.  Everything is integer-exact torch int64 arithmetic, so
the uniform stream is bit-identical on CPU and GPU; the Gaussians agree to the
last few ulps of the device's log/cos.

Workload recipes (the paper uses no public dataset; these stand in for its
lattice workloads):
  * gauge links  U = exp(i * eps * H), H a Gaussian traceless Hermitian matrix
    with density ~ exp(-Tr H^2), i.e. H = sum_a h^a T^a with h^a ~ N(0,1) for
    generators normalised Tr T^a T^b = delta/2;
  * optional Haar gauge transform  U(x,mu) -> g(x) U(x,mu) g(x+mu)^dag with
    g Haar-distributed in SU(N) (QR of a complex Ginibre matrix with the phase
    fix of Mezzadri 2007, then det -> 1);
  * spinors: complex Gaussian, Re and Im each N(0, 1/2) (unit variance).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF

# stream identifiers: one per kind of random field, so fields never overlap
STREAM_LINKS = 1
STREAM_GAUGE_TRANSFORM = 2
STREAM_SPINOR = 3
STREAM_DIRECTION = 4
STREAM_MOMENTUM = 5


def _mulhilo(a: torch.Tensor, m: int):
    """(hi, lo) 32-bit halves of a * m for a < 2^32 (int64), in 16-bit limbs so
    no intermediate exceeds 2^34."""
    a_lo = a & 0xFFFF
    a_hi = a >> 16
    m_lo = m & 0xFFFF
    m_hi = m >> 16
    ll = a_lo * m_lo
    lh = a_lo * m_hi
    hl = a_hi * m_lo
    hh = a_hi * m_hi
    mid = (ll >> 16) + (lh & 0xFFFF) + (hl & 0xFFFF)
    lo = ((mid & 0xFFFF) << 16) | (ll & 0xFFFF)
    hi = (hh + (lh >> 16) + (hl >> 16) + (mid >> 16)) & _MASK32
    return hi, lo


def philox4x32(counter, key):
    """Philox4x32-10 on int64 tensors holding 32-bit words.
    counter: tuple of 4 tensors (c0..c3); key: tuple of 2 python ints."""
    c0, c1, c2, c3 = counter
    k0, k1 = key[0] & _MASK32, key[1] & _MASK32
    for _ in range(10):
        hi0, lo0 = _mulhilo(c0, _M0)
        hi1, lo1 = _mulhilo(c2, _M1)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK32
        k1 = (k1 + _W1) & _MASK32
    return c0, c1, c2, c3


def uniforms(n: int, seed: int, stream: int, device="cpu") -> torch.Tensor:
    """n uniforms in (0, 1) as float64; element i comes from counter block i // 4."""
    nblk = (n + 3) // 4
    idx = torch.arange(nblk, dtype=torch.int64, device=device)
    zero = torch.zeros_like(idx)
    ctr = (idx & _MASK32, idx >> 32, zero + (stream & _MASK32), zero)
    words = torch.stack(philox4x32(ctr, (seed, seed >> 32)), dim=1).reshape(-1)[:n]
    return (words.to(torch.float64) + 0.5) * (1.0 / 4294967296.0)


def normals(n: int, seed: int, stream: int, device="cpu") -> torch.Tensor:
    """n standard normal variates (Box-Muller on pairs of uniforms), float64."""
    m = (n + 1) // 2
    u = uniforms(2 * m, seed, stream, device).reshape(m, 2)
    r = torch.sqrt(-2.0 * torch.log(u[:, 0]))
    th = 2.0 * math.pi * u[:, 1]
    return torch.stack((r * torch.cos(th), r * torch.sin(th)), dim=1).reshape(-1)[:n]


def gaussian_hermitian(count: int, N: int, seed: int, stream: int, device="cpu"):
    """count traceless Hermitian N x N matrices with density ~ exp(-Tr H^2)."""
    g = normals(count * N * N * 2, seed, stream, device).reshape(count, N, N, 2)
    G = torch.complex(g[..., 0], g[..., 1]) * math.sqrt(0.5)
    H = 0.5 * (G + G.conj().transpose(-1, -2))
    tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1) / N
    return H - tr[:, None, None] * torch.eye(N, dtype=H.dtype, device=device)


def expm_small(A: torch.Tensor, squarings: int = 6, order: int = 12) -> torch.Tensor:
    """exp(A) for a batch of small matrices: scaling and squaring with a
    truncated Taylor series (batched matmuls only, fast on any device)."""
    B = A * (1.0 / (1 << squarings))
    eye = torch.eye(A.shape[-1], dtype=A.dtype, device=A.device).expand_as(A)
    # Horner: I + B (I + B/2 (I + B/3 (...)))
    acc = eye.clone()
    for k in range(order, 0, -1):
        acc = eye + (B @ acc) * (1.0 / k)
    for _ in range(squarings):
        acc = acc @ acc
    return acc


def det_small(M: torch.Tensor) -> torch.Tensor:
    """determinant of a batch of N x N matrices (N <= 4) by cofactor expansion."""
    n = M.shape[-1]
    if n == 1:
        return M[..., 0, 0]
    if n == 2:
        return M[..., 0, 0] * M[..., 1, 1] - M[..., 0, 1] * M[..., 1, 0]
    d = torch.zeros(M.shape[:-2], dtype=M.dtype, device=M.device)
    for j in range(n):
        minor = torch.cat([M[..., 1:, :j], M[..., 1:, j + 1:]], dim=-1)
        d = d + ((-1) ** j) * M[..., 0, j] * det_small(minor)
    return d


def random_links(volume: int, N: int, eps: float, seed: int, device="cpu",
                 chunk: int = 1 << 21) -> torch.Tensor:
    """Gauge field U[V, 4, N, N] = exp(i eps H), complex128."""
    n = volume * 4
    out = torch.empty((n, N, N), dtype=torch.complex128, device=device)
    # the counter range is split by chunk so every element keeps its own counter
    per = N * N * 2
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        g = _normals_range(s * per, e * per, seed, STREAM_LINKS, device)
        g = g.reshape(e - s, N, N, 2)
        G = torch.complex(g[..., 0], g[..., 1]) * math.sqrt(0.5)
        H = 0.5 * (G + G.conj().transpose(-1, -2))
        tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1) / N
        H = H - tr[:, None, None] * torch.eye(N, dtype=H.dtype, device=device)
        out[s:e] = expm_small(1j * eps * H)
    return out.reshape(volume, 4, N, N)


def _normals_range(start: int, stop: int, seed: int, stream: int, device):
    """normals number start..stop-1 of the stream (start even)."""
    assert start % 2 == 0
    m0, m1 = start // 2, (stop + 1) // 2
    # uniform pair j uses uniforms 2j, 2j+1 -> counter block (2j)//4
    b0, b1 = (2 * m0) // 4, (2 * m1 + 3) // 4
    idx = torch.arange(b0, b1, dtype=torch.int64, device=device)
    zero = torch.zeros_like(idx)
    ctr = (idx & _MASK32, idx >> 32, zero + (stream & _MASK32), zero)
    words = torch.stack(philox4x32(ctr, (seed, seed >> 32)), dim=1).reshape(-1)
    words = words[2 * m0 - 4 * b0: 2 * m1 - 4 * b0]
    u = ((words.to(torch.float64) + 0.5) * (1.0 / 4294967296.0)).reshape(-1, 2)
    r = torch.sqrt(-2.0 * torch.log(u[:, 0]))
    th = 2.0 * math.pi * u[:, 1]
    z = torch.stack((r * torch.cos(th), r * torch.sin(th)), dim=1).reshape(-1)
    return z[start - 2 * m0: start - 2 * m0 + (stop - start)]


def haar_su_n(count: int, N: int, seed: int, stream: int = STREAM_GAUGE_TRANSFORM,
              device="cpu") -> torch.Tensor:
    """count Haar-random SU(N) matrices."""
    g = normals(count * N * N * 2, seed, stream, device).reshape(count, N, N, 2)
    Z = torch.complex(g[..., 0], g[..., 1]) * math.sqrt(0.5)
    # Gram-Schmidt on the columns = QR with a positive real diagonal of R,
    # which is the phase fix that makes Q Haar-distributed in U(N)
    cols = []
    for j in range(N):
        v = Z[:, :, j]
        for q in cols:
            v = v - (q.conj() * v).sum(-1, keepdim=True) * q
        v = v / torch.sqrt((v.conj() * v).real.sum(-1, keepdim=True))
        cols.append(v)
    Q = torch.stack(cols, dim=-1)
    det = det_small(Q)
    phase = torch.exp(-1j * torch.angle(det) / N)
    return Q * phase[:, None, None]


def shift(field: torch.Tensor, dims, mu: int, step: int) -> torch.Tensor:
    """field at x + step*mu_hat, for a field indexed by lexicographic site first."""
    T, X, Y, Z = dims
    f = field.reshape((T, X, Y, Z) + tuple(field.shape[1:]))
    f = torch.roll(f, shifts=-step, dims=mu)
    return f.reshape(field.shape)


def gauge_transform_links(U: torch.Tensor, g: torch.Tensor, dims) -> torch.Tensor:
    """U(x,mu) -> g(x) U(x,mu) g(x+mu)^dag."""
    out = torch.empty_like(U)
    for mu in range(4):
        gp = shift(g, dims, mu, +1)
        out[:, mu] = g @ U[:, mu] @ gp.conj().transpose(-1, -2)
    return out


def gaussian_spinor(nsites: int, D: int, seed: int, stream: int = STREAM_SPINOR,
                    device="cpu", nrhs: int = 1) -> torch.Tensor:
    """complex128 [nrhs, nsites, 4, D] (squeezed to [nsites, 4, D] for nrhs=1)."""
    n = nrhs * nsites * 4 * D
    g = normals(2 * n, seed, stream, device).reshape(n, 2) * math.sqrt(0.5)
    psi = torch.complex(g[:, 0], g[:, 1]).reshape(nrhs, nsites, 4, D)
    return psi[0] if nrhs == 1 else psi


# ---------------------------------------------------------------------------
# the five workloads (lattice, representation, mass, link recipe)
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    rep: str            # FUND / ADJ / SYM / ASYM / ASYM_REAL
    dims: tuple         # (T, X, Y, Z)
    m0: float
    eps: float          # link width: U = exp(i eps H)
    haar: bool = False  # random Haar gauge transform on top
    bc: tuple = (-1, 1, 1, 1)  # antiperiodic in time, periodic in space
    seed: int = 2503067210
    extra: dict = field(default_factory=dict)

    @property
    def volume(self):
        T, X, Y, Z = self.dims
        return T * X * Y * Z

    def links(self, device="cpu", dims=None):
        dims = dims or self.dims
        V = dims[0] * dims[1] * dims[2] * dims[3]
        U = random_links(V, self.N, self.eps, self.seed, device)
        if self.haar:
            g = haar_su_n(V, self.N, self.seed, device=device)
            U = gauge_transform_links(U, g, dims)
        return U


WORKLOADS = {
    # SU(2) adjoint 8^4, FP64 correctness configuration
    "su2_adj_8x8x8x8": Workload("su2_adj_8x8x8x8", 2, "ADJ", (8, 8, 8, 8), -0.2, 0.3,
                                seed=2503067211),
    # SU(3) two-index symmetric (sextet) 32^3 x 64
    "su3_sym_64x32x32x32": Workload("su3_sym_64x32x32x32", 3, "SYM", (64, 32, 32, 32), -0.3,
                                    0.4, haar=True, seed=2503067212),
    # SU(4) fundamental / antisymmetric 24^3 x 48 (+ uneven instances)
    "su4_fund_48x24x24x24": Workload("su4_fund_48x24x24x24", 4, "FUND", (48, 24, 24, 24),
                                     -0.25, 0.4, seed=2503067213),
    "su4_asym_48x24x24x24": Workload("su4_asym_48x24x24x24", 4, "ASYM", (48, 24, 24, 24),
                                     -0.25, 0.4, seed=2503067213),
    # the same SU(4) 2AS workload with the links in the real basis (stored real)
    "su4_asym_real_48x24x24x24": Workload("su4_asym_real_48x24x24x24", 4, "ASYM_REAL", (48, 24, 24, 24),
                                          -0.25, 0.4, seed=2503067213),
    # SU(4) adjoint (D_R = 15) and symmetric (D_R = 10) 24^3 x 48: the colour-parallel kernel
    "su4_adj_48x24x24x24": Workload("su4_adj_48x24x24x24", 4, "ADJ", (48, 24, 24, 24), -0.25, 0.4,
                                    seed=2503067216),
    "su4_sym_48x24x24x24": Workload("su4_sym_48x24x24x24", 4, "SYM", (48, 24, 24, 24), -0.25, 0.4,
                                    seed=2503067217),
    # SU(5) fundamental 24^3 x 48: the colour-parallel kernel with an odd D_R
    "su5_fund_48x24x24x24": Workload("su5_fund_48x24x24x24", 5, "FUND", (48, 24, 24, 24),
                                     -0.1, 0.4, seed=2503067219),
    # SU(8) fundamental 24^3 x 48: the colour-parallel (large-N) kernel
    "su8_fund_48x24x24x24": Workload("su8_fund_48x24x24x24", 8, "FUND", (48, 24, 24, 24),
                                     -0.1, 0.4, seed=2503067218),
    # SU(3) sextet 16^3 x 32, force / differentiation configuration
    "su3_sym_32x16x16x16": Workload("su3_sym_32x16x16x16", 3, "SYM", (32, 16, 16, 16), -0.3,
                                    0.4, seed=2503067214),
    # SU(3) sextet 32^4: the same kernel on a lattice small enough for profiler captures
    "su3_sym_32x32x32x32": Workload("su3_sym_32x32x32x32", 3, "SYM", (32, 32, 32, 32), -0.3,
                                    0.4, haar=True, seed=2503067212),
    # SU(3) adjoint 32^4: profiler-sized lattice of the adjoint kernels
    "su3_adj_32x32x32x32": Workload("su3_adj_32x32x32x32", 3, "ADJ", (32, 32, 32, 32), -0.35, 0.5,
                                    seed=2503067215),
    # SU(3) adjoint 64^3 x 128, stored vs rebuilt links
    "su3_adj_128x64x64x64": Workload("su3_adj_128x64x64x64", 3, "ADJ", (128, 64, 64, 64),
                                     -0.35, 0.5, seed=2503067215),
}

# uneven instances solved together with the 24^3 x 48 lattice (zipped masses)
UNEVEN_INSTANCES = [((8, 8, 8, 8), -0.1), ((12, 12, 12, 12), -0.25), ((32, 16, 16, 16), -0.4)]
