"""The five seeded QAOA Max-Cut workloads and their angle draws.

Each workload fixes the graph family (n vertices, degree d, seed), the QAOA
depth p, the angles, the ordering scheme, the element type and the network
form.  Angles are either fixed or drawn uniformly with gamma in [0, pi) and
beta in [0, pi/2) from a SplitMix64 stream: gamma_1..gamma_p first, then
beta_1..beta_p.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

from .graphs import random_regular_graph
from .rng import SplitMix64


def qaoa_angles(p: int, seed: int):
    """(gammas, betas) for depth p: gamma ~ U[0, pi), beta ~ U[0, pi/2)."""
    rng = SplitMix64(seed)
    gammas = [math.pi * rng.uniform() for _ in range(p)]
    betas = [0.5 * math.pi * rng.uniform() for _ in range(p)]
    return gammas, betas


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    p: int
    graph_seed: int
    ordering: str          # "stoch" or "lg"
    dtype: str             # "c128", "c64", "split_bf16"
    diag: bool             # diagonal (hyperedge) ZZ gates instead of rank-4
    lightcone: bool        # per-edge reverse light cone
    gammas: tuple = field(default=())
    betas: tuple = field(default=())
    angle_seed: int | None = None
    want_grad: bool = False
    restarts: int = 8      # randomised min-fill runs of the LG ordering
    description: str = ""

    def graph(self):
        return random_regular_graph(self.n, self.d, self.graph_seed)

    def angles(self):
        if self.angle_seed is None:
            return list(self.gammas), list(self.betas)
        return qaoa_angles(self.p, self.angle_seed)


WORKLOADS = {
    "qaoa_p1_n12_d3": Workload(
        "qaoa_p1_n12_d3", n=12, d=3, p=1, graph_seed=0, ordering="stoch",
        dtype="c128", diag=False, lightcone=True, gammas=(0.7,), betas=(0.4,),
        description="p=1, 3-regular, 12 vertices, gamma=0.7, beta=0.4, "
                    "rank-4 ZZ tensors, stochastic ordering, complex128"),
    "qaoa_p1_n50_d3": Workload(
        "qaoa_p1_n50_d3", n=50, d=3, p=1, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=True, angle_seed=0,
        description="p=1, 3-regular, 50 vertices / 75 edges, random angles, "
                    "line-graph ordering, complex64"),
    "qaoa_p2_n100_d5": Workload(
        "qaoa_p2_n100_d5", n=100, d=5, p=2, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=True, angle_seed=0,
        description="p=2, 5-regular, 100 vertices / 250 edges, batched "
                    "light-cone networks"),
    "qaoa_p3_n60_d4": Workload(
        "qaoa_p3_n60_d4", n=60, d=4, p=3, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=True, angle_seed=0, want_grad=True, restarts=1024,
        description="p=3, 4-regular, 60 vertices / 120 edges, value and "
                    "gradient"),
    "qaoa_p1_n20_d7": Workload(
        "qaoa_p1_n20_d7", n=20, d=7, p=1, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=False, angle_seed=0,
        description="p=1, 7-regular, 20 vertices, full un-reduced networks"),
    "qaoa_p1_n24_d7": Workload(
        "qaoa_p1_n24_d7", n=24, d=7, p=1, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=False, angle_seed=0,
        description="p=1, 7-regular, 24 vertices, full un-reduced networks"),
    "qaoa_p1_n26_d7": Workload(
        "qaoa_p1_n26_d7", n=26, d=7, p=1, graph_seed=0, ordering="lg",
        dtype="c64", diag=True, lightcone=False, angle_seed=0,
        description="p=1, 7-regular, 26 vertices, full un-reduced networks"),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
