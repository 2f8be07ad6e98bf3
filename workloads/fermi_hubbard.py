"""Spinful Fermi-Hubbard brickwall circuits (seeded synthetic workloads).

Conventions (paper Sec. "Model system and circuit topology", Eq. sfFH, and the
state-vector layout of Sec. "Details of the state vector simulation"):

* ``n = 2L`` qubits; qubit ``j`` is (site j, spin up), qubit ``L + j`` is
  (site j, spin down); qubit 0 is the most significant bit of an amplitude
  index.
* A gate on the listed pair ``(a, b)`` is a 4x4 complex matrix whose local
  index is ``2 * bit_a + bit_b``.
* The circuit is the sequential list ``G_1, ..., G_g`` with ``G_1`` applied
  first (``W = G_g ... G_1``); the brickwall is sequentialised layer by layer,
  gates inside a layer sorted by their first qubit (paper Fig.
  brickwall_to_sequential).
* Layer kinds: ``A`` even hopping bonds ``(2k, 2k+1)`` of both spin chains,
  ``B`` odd hopping bonds ``(2k+1, 2k+2)``, ``C`` on-site pairs ``(j, L+j)``;
  a depth-``d`` circuit follows the cyclic pattern ``A B C B`` cut to ``d``
  layers.  A periodic chain adds the wrap bond ``(L-1, 0)`` to ``B`` (``A``
  when ``L`` is odd is not used by any workload here).
* Initial gates are the two-site Trotter factors ``exp(-i tau h)`` (paper Eq.
  for ``exp(-i t h_loc)``), times ``expm(sigma * A)`` with ``A`` a seeded
  Gaussian skew-Hermitian matrix (masked to the parity pattern for
  parity-structured circuits).

Random numbers come only from ``numpy.random.default_rng(seed)`` on the host.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

# Local two-qubit index 2*bit_a + bit_b: even parity {0, 3}, odd parity {1, 2}
# (paper Eq. paritygatematrix: nonzeros g11, g14, g41, g44, g22, g23, g32, g33).
_PARITY = np.array([0, 1, 1, 0])


def parity_mask() -> np.ndarray:
    """Boolean 4x4 mask of the parity-conserving gate pattern."""
    return _PARITY[:, None] == _PARITY[None, :]


def layer_pattern(depth: int) -> List[str]:
    """Layer kinds of a depth-``depth`` brickwall: ``ABCB`` repeated, cut."""
    cyc = "ABCB"
    return [cyc[i % 4] for i in range(depth)]


def brickwall_layers(L: int, depth: int, periodic: bool = False):
    """Qubit pairs of every layer, as a list of ``(kind, [(a, b), ...])``."""
    layers = []
    for kind in layer_pattern(depth):
        pairs: List[Tuple[int, int]] = []
        if kind == "C":
            pairs = [(j, L + j) for j in range(L)]
        else:
            start = 0 if kind == "A" else 1
            for off in (0, L):  # up chain, then down chain
                for s in range(start, L - 1, 2):
                    pairs.append((off + s, off + s + 1))
                if periodic and kind == "B" and L % 2 == 0 and L > 2:
                    pairs.append((off + L - 1, off + 0))
            pairs.sort(key=lambda p: p[0])
        layers.append((kind, pairs))
    return layers


def trotter_times(depth: int, t: float) -> List[float]:
    """Per-layer evolution times of the Trotter initialisation.

    ``depth = 4r + 1``: ``r`` merged Strang steps of ``dt = t / r`` (outer ``A``
    layers ``dt/2``, inner ``A`` ``dt``, every ``B`` ``dt/2``, every ``C``
    ``dt``).  Otherwise each kind's total time ``t`` is split evenly over its
    occurrences (a first-order product formula).
    """
    kinds = layer_pattern(depth)
    if depth % 4 == 1 and depth >= 5:
        r = (depth - 1) // 4
        dt = t / r
        out = []
        for i, k in enumerate(kinds):
            if k == "A":
                out.append(dt / 2 if i in (0, depth - 1) else dt)
            elif k == "B":
                out.append(dt / 2)
            else:
                out.append(dt)
        return out
    counts = {k: kinds.count(k) for k in "ABC"}
    return [t / counts[k] for k in kinds]


def trotter4_times(t: float) -> List[float]:
    """21 layer times of a 4th-order Suzuki step for the 3-term split A + B + C.

    ``S4(t) = S2(p t)^2 S2((1 - 4p) t) S2(p t)^2`` with ``p = 1 / (4 - 4^(1/3))``
    and the nested Strang step ``S2(s) = A(s/2) B(s/2) C(s) B(s/2) A(s/2)``;
    adjacent ``A`` factors of consecutive steps merge, leaving
    ``5 * 4 + 1 = 21`` layers ``ABCB...A``.
    """
    p = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
    steps = [p, p, 1.0 - 4.0 * p, p, p]
    out = [steps[0] * t / 2]
    for k, sk in enumerate(steps):
        out += [sk * t / 2, sk * t, sk * t / 2]
        nxt = steps[k + 1] * t / 2 if k + 1 < len(steps) else 0.0
        out.append(sk * t / 2 + nxt)
    return out


def trotter_gate(kind: str, tau: float, J: float, U: float) -> np.ndarray:
    """Closed-form ``exp(-i tau h)`` for a hopping (A/B) or on-site (C) pair."""
    g = np.zeros((4, 4), dtype=np.complex128)
    if kind in ("A", "B"):
        c, s = np.cos(J * tau), np.sin(J * tau)
        g[0, 0] = 1.0
        g[1, 1] = c
        g[1, 2] = 1j * s
        g[2, 1] = 1j * s
        g[2, 2] = c
        g[3, 3] = 1.0
    else:
        g[0, 0] = g[1, 1] = g[2, 2] = 1.0
        g[3, 3] = np.exp(-1j * U * tau)
    return g


def _noise(rng: np.random.Generator, sigma: float, parity: bool) -> np.ndarray:
    X = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    A = 0.5 * (X - X.conj().T)
    if parity:
        A = A * parity_mask()
    return scipy.linalg.expm(sigma * A)


@dataclass
class Problem:
    """One circuit-optimisation instance (all arrays plain numpy)."""

    L: int
    depth: int
    t: float
    J: float
    U: float
    periodic: bool
    structure: int  # 0 general 4x4 gates, 1 parity-conserving gates
    pairs: np.ndarray  # [g, 2] int32
    param_of: np.ndarray  # [g] int32
    gates: np.ndarray  # [n_params, 4, 4] complex128
    kinds: List[str] = field(default_factory=list)  # layer kind per gate
    model: int = 0  # 0 spinful chain (n = 2L), 1 spinless chain (n = L)

    @property
    def n(self) -> int:
        return 2 * self.L if self.model == 0 else self.L

    @property
    def n_gates(self) -> int:
        return int(self.pairs.shape[0])

    @property
    def n_params(self) -> int:
        return int(self.gates.shape[0])


def make_problem(L: int, depth: int, t: float, U: float = 4.0, J: float = 1.0,
                 seed: int = 0, structure: int = 0, tied: bool = False,
                 periodic: bool = False, sigma: float = 1e-2, order: int = 2) -> Problem:
    """Trotter-initialised brickwall for the spinful chain with seeded noise.

    ``tied``: one parameter gate per layer (translation-invariant ansatz,
    paper Sec. "Brick wall circuit layout"); otherwise one per gate.
    ``order = 4`` (with ``depth = 21``): the 4th-order Suzuki initialisation
    the paper uses for its convergence comparison.
    """
    rng = np.random.default_rng(seed)
    layers = brickwall_layers(L, depth, periodic)
    if order == 4:
        if depth != 21:
            raise ValueError("the 4th-order initialisation has 21 layers")
        taus = trotter4_times(t)
    else:
        taus = trotter_times(depth, t)
    pairs, param_of, gates, kinds = [], [], [], []
    for li, ((kind, lp), tau) in enumerate(zip(layers, taus)):
        if tied and lp:
            gates.append(trotter_gate(kind, tau, J, U) @ _noise(rng, sigma, structure == 1))
        for p in lp:
            pairs.append(p)
            kinds.append(kind)
            if tied:
                param_of.append(len(gates) - 1)
            else:
                gates.append(trotter_gate(kind, tau, J, U) @ _noise(rng, sigma, structure == 1))
                param_of.append(len(gates) - 1)
    return Problem(L=L, depth=depth, t=t, J=J, U=U, periodic=periodic,
                   structure=structure,
                   pairs=np.asarray(pairs, dtype=np.int32).reshape(-1, 2),
                   param_of=np.asarray(param_of, dtype=np.int32),
                   gates=np.asarray(gates, dtype=np.complex128).reshape(-1, 4, 4),
                   kinds=kinds)


def random_directions(n_params: int, k: int, seed: int) -> np.ndarray:
    """Raw Gaussian complex 4x4 matrices ``[k, n_params, 4, 4]``.

    Both the CUDA path and the oracle project them onto the tangent space
    themselves before use.
    """
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((k, n_params, 4, 4))
            + 1j * rng.standard_normal((k, n_params, 4, 4)))


def random_unitary(dim: int, seed: int) -> np.ndarray:
    """Haar-distributed ``dim x dim`` unitary (QR of a complex Gaussian
    matrix with the phases of R's diagonal moved into Q), a dense target for
    tests of targets that are not a chain's time evolution."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))


# Spinless chain (paper Eq. slFH_qubit) -----------------------------------------

def spinless_layers(L: int, depth: int, periodic: bool = False):
    """Even bonds ``E`` = (2k, 2k+1), odd bonds ``O`` = (2k+1, 2k+2) (plus the
    wrap bond (L-1, 0) of an even periodic chain), alternating ``EOEO...``."""
    layers = []
    for i in range(depth):
        kind = "E" if i % 2 == 0 else "O"
        start = 0 if kind == "E" else 1
        pairs = [(s, s + 1) for s in range(start, L - 1, 2)]
        if periodic and kind == "O" and L % 2 == 0 and L > 2:
            pairs.append((L - 1, 0))
        layers.append((kind, pairs))
    return layers


def spinless_times(depth: int, t: float) -> List[float]:
    """Odd depth 2r+1: r merged Strang steps (outer E layers dt/2, inner E
    and all O layers dt, dt = t/r); otherwise t split evenly per kind."""
    if depth % 2 == 1 and depth >= 3:
        r = (depth - 1) // 2
        dt = t / r
        return [dt / 2 if i in (0, depth - 1) else dt for i in range(depth)]
    kinds = ["E" if i % 2 == 0 else "O" for i in range(depth)]
    return [t / kinds.count(k) for k in kinds]


def spinless_gate(tau: float, J: float, U: float) -> np.ndarray:
    """The paper's closed form of ``exp(-i tau h_loc)`` (hop + U n n)."""
    g = trotter_gate("A", tau, J, U)
    g[3, 3] = np.exp(-1j * U * tau)
    return g


def make_spinless_problem(L: int, depth: int, t: float, U: float = 2.0, J: float = 1.0, seed: int = 0,
                          structure: int = 0, tied: bool = False, periodic: bool = False,
                          sigma: float = 1e-2) -> Problem:
    """Trotter-initialised brickwall for the spinless hard-core-boson chain."""
    rng = np.random.default_rng(seed)
    pairs, param_of, gates, kinds = [], [], [], []
    for (kind, lp), tau in zip(spinless_layers(L, depth, periodic), spinless_times(depth, t)):
        if tied and lp:
            gates.append(spinless_gate(tau, J, U) @ _noise(rng, sigma, structure == 1))
        for p in lp:
            pairs.append(p)
            kinds.append(kind)
            if not tied:
                gates.append(spinless_gate(tau, J, U) @ _noise(rng, sigma, structure == 1))
            param_of.append(len(gates) - 1)
    return Problem(L=L, depth=depth, t=t, J=J, U=U, periodic=periodic, structure=structure,
                   pairs=np.asarray(pairs, dtype=np.int32).reshape(-1, 2),
                   param_of=np.asarray(param_of, dtype=np.int32),
                   gates=np.asarray(gates, dtype=np.complex128).reshape(-1, 4, 4), kinds=kinds, model=1)


# Named workloads ------------------------------------------------------------

def config_problem(name: str, structure: Optional[int] = None) -> Problem:
    """The named instances used by tests and the benchmark.

    ``small``   n=8 (4 sites), 5 layers ABCBA, t=0.25, general, seed 101
    ``tied12``  n=12 (6 sites), 9 layers, t=0.5, one gate per layer, parity,
                seed 201
    ``n14``     n=14 (7 sites), 7 layers, t=0.5, general, seed 401
    ``n16``     n=16 (8 sites), 11 layers ABCBABCBABC, t=0.5, general (or
                parity with ``structure=1``), seed 1601
    """
    if name == "small":
        return make_problem(4, 5, 0.25, seed=101, structure=structure or 0)
    if name == "tied12":
        return make_problem(6, 9, 0.5, seed=201, tied=True,
                            structure=1 if structure is None else structure)
    if name == "n14":
        return make_problem(7, 7, 0.5, seed=401, structure=structure or 0)
    if name == "n16":
        return make_problem(8, 11, 0.5, seed=1601, structure=structure or 0)
    raise KeyError(name)


def batch_problems(count: int, seed: int = 301, sizes: Sequence[int] = (4, 5, 6),
                   depths: Sequence[int] = (3, 5, 7, 9)) -> List[Problem]:
    """Independent problems of uneven size: L in ``sizes`` (n = 2L),
    depth in ``depths``, t ~ U[0.1, 1], U ~ U[2, 8]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        L = int(rng.choice(sizes))
        d = int(rng.choice(depths))
        t = float(rng.uniform(0.1, 1.0))
        U = float(rng.uniform(2.0, 8.0))
        out.append(make_problem(L, d, t, U=U, seed=int(rng.integers(1 << 30))))
    return out
