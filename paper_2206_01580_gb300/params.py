"""FCHL19 hyperparameters as the library consumes them.

The values are the optimised parameters of the paper's table in the
Computational Details section: column "E" for energy-only learning, column
"E + F" for energy and force learning. n2 and n3 can be overridden (the
synthetic workloads use n2 = 24, n3 = 22, giving a 780-wide representation).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

TABLE = {
    "E": dict(n2=23, n3=22, eta2=0.27, eta3=5.6, N2=2.78, N3=2.1, c3=60.1, zeta=math.pi, rcut=6.0),
    "EF": dict(n2=24, n3=20, eta2=0.32, eta3=2.7, N2=1.8, N3=0.57, c3=13.4, zeta=math.pi, rcut=6.0),
}


@dataclass(frozen=True)
class FCHL19Params:
    n_el: int = 5
    n2: int = 24
    n3: int = 22
    nfourier: int = 1
    eta2: float = 0.27
    eta3: float = 5.6
    N2: float = 2.78
    N3: float = 2.1
    c3: float = 60.1
    zeta: float = math.pi
    rcut: float = 6.0

    @property
    def rep_dim(self) -> int:
        return self.n_el * self.n2 + self.n_el * (self.n_el + 1) // 2 * self.n3 * 2

    def with_sizes(self, n2: int, n3: int) -> "FCHL19Params":
        return replace(self, n2=n2, n3=n3)


def from_table(column: str, n2: int | None = None, n3: int | None = None, n_el: int = 5) -> FCHL19Params:
    t = dict(TABLE[column])
    if n2 is not None:
        t["n2"] = n2
    if n3 is not None:
        t["n3"] = n3
    return FCHL19Params(n_el=n_el, **t)
