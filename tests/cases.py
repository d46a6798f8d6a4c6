"""Seeded test cases shared by the GPU parity tests: the same inputs for the CUDA library and the oracle."""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_mass(name: str) -> float:
    with open(os.path.join(HERE, "golden", "masses.json")) as f:
        return json.load(f)["masses"][name]["m0"]


@dataclass
class Case:
    dims: tuple
    levels: int
    agg: tuple                 # per level l < L-1
    n_tv: tuple                # per level l < L-1
    sap: tuple                 # per level l < L-1
    m0: float = -0.2
    csw: float = 1.0
    bc_t: int = -1
    eps: float = 0.4
    seed: int = 0
    mr_steps: int = 3
    nu: int = 2
    mu: int = 0
    n_inv: int = 0
    eta_passes: int = 0
    outer_restart: int = 10
    coarse_restart: int = 50
    max_rhs: int = 1
    extra: dict = field(default_factory=dict)

    def level_dims(self):
        out = [tuple(self.dims)]
        for l in range(self.levels - 1):
            out.append(tuple(d // a for d, a in zip(out[-1], self.agg[l])))
        return out

    def gauge(self):
        return synth.su3_field(self.dims, self.eps, self.seed)

    def random_tv(self):
        ld = self.level_dims()
        out = [synth.random_fields(self.n_tv[0], ld[0], 12, self.seed + 100)]
        for l in range(1, self.levels - 1):
            extra = max(0, self.n_tv[l] - self.n_tv[l - 1])
            out.append(synth.random_fields(extra, ld[l], 2 * self.n_tv[l - 1], self.seed + 100 + l)
                       if extra else None)
        return out

    def gpu_params(self, precision=0):
        import paper_1307_6101_gb300 as dd
        kw = dict(levels=self.levels, agg=list(self.agg), n_tv=list(self.n_tv), sap_block=list(self.sap),
                  mr_steps=self.mr_steps, nu=self.nu, mu=self.mu, n_inv=self.n_inv,
                  eta_passes=self.eta_passes, outer_restart=self.outer_restart,
                  coarse_restart=self.coarse_restart, precision=precision, max_rhs=self.max_rhs)
        kw.update(self.extra)
        return dd.ddamg_default_params(**kw)

    def oracle_params(self):
        from oracle.multigrid import Params
        kw = dict(levels=self.levels, agg=tuple(self.agg), n_tv=tuple(self.n_tv),
                  sap_block=tuple(self.sap) + (None,), mr_steps=self.mr_steps, nu=self.nu, mu=self.mu,
                  n_inv=self.n_inv, eta_passes=self.eta_passes, outer_restart=self.outer_restart,
                  coarse_restart=self.coarse_restart)
        for k in ("kcycle_len", "kcycle_cycles", "kcycle_tol", "coarse_tol", "coarse_cycles"):
            if k in self.extra:
                kw[k] = self.extra[k]
        if "outer_max_cycles" in self.extra:
            kw["outer_max_cycles"] = self.extra["outer_max_cycles"]
        return Params(**kw)

    def gpu(self, precision=0, U=None, tv=None):
        import paper_1307_6101_gb300 as dd
        U = self.gauge() if U is None else U
        tv = self.random_tv() if tv is None else tv
        return dd.ddamg_setup(U, self.dims, self.bc_t, self.m0, self.csw, self.gpu_params(precision), tv)

    def oracle(self, U=None, tv=None):
        from oracle.wilson import WilsonOp
        from oracle.multigrid import Hierarchy
        U = self.gauge() if U is None else U
        tv = self.random_tv() if tv is None else tv
        op = WilsonOp.build(U, self.m0, self.csw, self.bc_t)
        return Hierarchy(op, self.oracle_params()).setup(tv)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# lattices used by the parity tests
SMALL2 = dict(dims=(4, 4, 4, 4), levels=2, agg=((2, 2, 2, 2),), n_tv=(3,), sap=((2, 2, 2, 2),))
RAGGED2 = dict(dims=(4, 6, 6, 4), levels=2, agg=((2, 3, 3, 2),), n_tv=(4,), sap=((2, 3, 3, 2),))
THREE = dict(dims=(8, 4, 4, 4), levels=3, agg=((2, 2, 2, 2), (2, 1, 1, 1)), n_tv=(4, 6),
             sap=((2, 2, 2, 2), (2, 2, 2, 2)))
# odd extents: level-1 SAP blocks widen to (2, 3, 3, 3) (not nested with the 2^4 aggregates)
# and the coarsest lattice (2, 3, 3, 3) is solved by plain GMRES
ODD3 = dict(dims=(8, 12, 12, 12), levels=3, agg=((2, 2, 2, 2), (2, 2, 2, 2)), n_tv=(4, 5),
            sap=((2, 2, 2, 2), (2, 2, 2, 2)))
# four levels (the structure of the 48^3x96 workload at a small size): aggregates 2^4 three
# times; the coarsest lattice (2, 1, 1, 1) has odd extents and is solved by plain GMRES
FOUR = dict(dims=(16, 8, 8, 8), levels=4, agg=((2, 2, 2, 2), (2, 2, 2, 2), (2, 2, 2, 2)), n_tv=(4, 5, 5),
            sap=((2, 2, 2, 2), (2, 2, 2, 2), (2, 2, 2, 2)))
# 4^4 SAP blocks on the fine level (the block of the three-level workloads), with 4^4 aggregates so
# that the SAP block is the contiguous inner tile; SAP4W's blocks span the whole t and y extents, so
# hops through those lattice boundaries (antiperiodic in t) wrap inside the block
SAP4 = dict(dims=(8, 8, 8, 8), levels=2, agg=((4, 4, 4, 4),), n_tv=(3,), sap=((4, 4, 4, 4),))
SAP4W = dict(dims=(4, 8, 4, 8), levels=2, agg=((4, 4, 4, 4),), n_tv=(3,), sap=((4, 4, 4, 4),))
# Krylov vectors long enough for the cluster-split Arnoldi step of the device-driven (F)GMRES:
# BIG2's coarsest Schur vectors have 128 * 32 = 4096 entries, BIG3's level-1 vectors 256 * 16
BIG2 = dict(dims=(8, 8, 8, 8), levels=2, agg=((2, 2, 2, 2),), n_tv=(16,), sap=((2, 2, 2, 2),))
BIG3 = dict(dims=(8, 8, 8, 8), levels=3, agg=((2, 2, 2, 2), (2, 2, 2, 2)), n_tv=(8, 10),
            sap=((2, 2, 2, 2), (2, 2, 2, 2)))
# level-1 SAP blocks widened to 2x3x3x3 sites of 56 dof (3024 rows, not nested in the 2^4
# aggregates): the one-CTA-per-block coarse SAP kernel at eight rows per thread
ODDBIG = dict(dims=(8, 12, 12, 12), levels=3, agg=((2, 2, 2, 2), (2, 2, 2, 2)), n_tv=(28, 28),
              sap=((2, 2, 2, 2), (2, 2, 2, 2)))
# the two-level FP64 workload (8^4, eps 0.3, csw 0, aggregates 4^4, 8 test vectors, SAP 2^4)
C1 = dict(dims=(8, 8, 8, 8), levels=2, agg=((4, 4, 4, 4),), n_tv=(8,), sap=((2, 2, 2, 2),), eps=0.3, csw=0.0,
          mr_steps=4, nu=3, n_inv=3, eta_passes=3, outer_restart=25)
