"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only fixes workload shapes
and draws FP64 parameter vectors from numpy's ``default_rng(seed)``.  Random
numbers that the method itself draws (initial spins, proposals, uniforms) are
produced on each side by its own Philox4x32-10 implementation.

Parameter vector layouts (FP64, flat):
  RBM   : [a (N) | b (M) | W (M x N, row-major: W[j, i] couples hidden j to site i)]
  dense : [W1 (H1 x N) | b1 (H1) | W2 (H2 x H1) | b2 | ... | w_out (H_L) | b_out (1)]
"""
from dataclasses import dataclass, field
import numpy as np

SEED_BASE = 20260000


@dataclass(frozen=True)
class Lattice:
    Lx: int
    Ly: int = 1          # Ly == 1: a 1D periodic chain of Lx sites

    @property
    def n_sites(self):
        return self.Lx * self.Ly


@dataclass(frozen=True)
class Hamiltonian:
    kind: str            # "tfim" or "heisenberg"
    lattice: Lattice
    J1: float = 1.0
    J2: float = 0.0
    h: float = 0.0
    marshall: bool = False


@dataclass(frozen=True)
class Workload:
    name: str
    ham: Hamiltonian
    model: str                      # "rbm" or "dense"
    n_hidden: int = 0               # RBM M
    widths: tuple = ()              # dense hidden widths
    weight_sigma: float = 0.0       # RBM weights ~ N(0, sigma^2)
    n_chains: int = 0
    n_sweeps: int = 0
    burn_in: int = 0
    dtypes: tuple = ("f32",)
    seed: int = SEED_BASE
    extra: dict = field(default_factory=dict)


def rbm_n_params(n, m):
    return n + m + m * n


def dense_n_params(n, widths):
    p, fan = 0, n
    for w in widths:
        p += w * fan + w
        fan = w
    return p + fan + 1


def rbm_params(n, m, sigma, seed):
    """a, b, W ~ N(0, sigma^2) i.i.d. in FP64, flattened as [a | b | W]."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=rbm_n_params(n, m)).astype(np.float64)


def complex_rbm_params(n, m, sigma, seed):
    """Complex a, b, W: the real parts are rbm_params(n, m, sigma, seed), the imaginary parts
    N(0, sigma^2) i.i.d. from seed + 1 (complex128, order [a | b | W])."""
    im = np.random.default_rng(seed + 1).normal(0.0, sigma, size=rbm_n_params(n, m))
    return rbm_params(n, m, sigma, seed) + 1j * im


def dense_params(n, widths, seed, bias_sigma=0.0):
    """He initialisation: W_l ~ N(0, 2 / fan_in); biases ~ N(0, bias_sigma^2) (0 by default)."""
    rng = np.random.default_rng(seed)
    parts, fan = [], n
    for w in widths:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan), size=w * fan))
        parts.append(rng.normal(0.0, bias_sigma, size=w) if bias_sigma > 0 else np.zeros(w))
        fan = w
    parts.append(rng.normal(0.0, np.sqrt(2.0 / fan), size=fan))
    parts.append(rng.normal(0.0, bias_sigma, size=1) if bias_sigma > 0 else np.zeros(1))
    return np.concatenate(parts).astype(np.float64)


def rescnn_params(n_filters, n_blocks, seed, gamma_sigma=0.25, bias_sigma=0.1):
    """ResCNN (App. H) parameters in the oracle's flat order: kernels ~ N(0, 1 / fan_in) with
    fan_in = 9 x input channels; conv biases and LN shifts ~ N(0, bias_sigma^2); LN scales
    ~ 1 + N(0, gamma_sigma^2) (scales all equal to 1 would make the summed output constant)."""
    rng = np.random.default_rng(seed)
    F = n_filters
    parts = [rng.normal(0.0, np.sqrt(1.0 / 9.0), size=9 * F), rng.normal(0.0, bias_sigma, size=F)]
    for _ in range(n_blocks):
        parts += [1.0 + rng.normal(0.0, gamma_sigma, size=F), rng.normal(0.0, bias_sigma, size=F)]
        for _ in range(2):
            parts += [rng.normal(0.0, np.sqrt(1.0 / (9.0 * F)), size=9 * F * F), rng.normal(0.0, bias_sigma, size=F)]
    parts += [1.0 + rng.normal(0.0, gamma_sigma, size=F), rng.normal(0.0, bias_sigma, size=F)]
    return np.concatenate(parts).astype(np.float64)


# The five workloads the build is measured and checked on.
TFIM_1D_N16 = Workload(
    name="tfim1d_n16_rbm_a1", ham=Hamiltonian("tfim", Lattice(16), J1=1.0, h=1.0),
    model="rbm", n_hidden=16, weight_sigma=0.01, n_chains=1024, n_sweeps=100, burn_in=10,
    dtypes=("f32",), seed=SEED_BASE + 1)

TFIM_2D_10x10 = Workload(
    name="tfim2d_10x10_rbm_a4", ham=Hamiltonian("tfim", Lattice(10, 10), J1=1.0, h=3.04),
    model="rbm", n_hidden=400, weight_sigma=0.05, n_chains=16384, n_sweeps=500, burn_in=50,
    dtypes=("f32", "bf16", "f16"), seed=SEED_BASE + 2,
    extra={"small_case": Lattice(4, 4)})

HEIS_2D_10x10 = Workload(
    name="heis2d_10x10_dense_100_400_400_1",
    ham=Hamiltonian("heisenberg", Lattice(10, 10), J1=1.0, J2=0.0, marshall=True),
    model="dense", widths=(400, 400), n_chains=8192, n_sweeps=51, burn_in=50,
    dtypes=("bf16",), seed=SEED_BASE + 3)

J1J2_2D_16x16 = Workload(
    name="j1j2_2d_16x16_dense_256_1024x3_1",
    ham=Hamiltonian("heisenberg", Lattice(16, 16), J1=1.0, J2=0.5, marshall=True),
    model="dense", widths=(1024, 1024, 1024), n_chains=65536, n_sweeps=200, burn_in=20,
    dtypes=("fp8", "bf16"), seed=SEED_BASE + 5, extra={"minsr_samples": 4096})


RESCNN_2D_10x10 = Workload(
    name="rescnn_tfim2d_10x10_4blocks_16filters",
    ham=Hamiltonian("tfim", Lattice(10, 10), J1=1.0, h=3.04), model="rescnn",
    n_chains=8192, n_sweeps=10, burn_in=2, dtypes=("f16", "bf16", "f32"), seed=SEED_BASE + 6,
    extra={"filters": 16, "blocks": 4, "small_case": Lattice(4, 4)})


def batched_tfim_instances(seed=SEED_BASE + 4, n_instances=48):
    """48 independent TFIM problems, 1D and 2D, N in {36, 64, 100, 144, 196, 256},
    h ~ U[0.5, 4], alpha in {1, 2, 4}, chains log-uniform in [256, 8192]."""
    rng = np.random.default_rng(seed)
    sizes = [36, 64, 100, 144, 196, 256]
    out = []
    for k in range(n_instances):
        n = sizes[k % len(sizes)]
        two_d = bool(rng.integers(0, 2))
        lat = Lattice(int(round(np.sqrt(n))), int(round(np.sqrt(n)))) if two_d else Lattice(n)
        alpha = int(rng.choice([1, 2, 4]))
        chains = int(np.exp(rng.uniform(np.log(256), np.log(8192))))
        h = float(rng.uniform(0.5, 4.0))
        out.append(Workload(
            name=f"inst{k:02d}", ham=Hamiltonian("tfim", lat, J1=1.0, h=h), model="rbm",
            n_hidden=alpha * n, weight_sigma=0.05 / np.sqrt(alpha), n_chains=chains,
            n_sweeps=20, burn_in=2, dtypes=("f16",), seed=seed * 100 + k))
    return out
