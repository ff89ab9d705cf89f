"""Named workloads: the problem sizes, media, right-hand sides, preconditioners and training
recipes of the solver's standard cases, so that a run is set up from one name.

Each preset is plain data (no GPU work here).  `helmholtz_overrides` gives the helm_desc
fields for lib.Helmholtz, `medium` and `rhs` build the seeded inputs.  Settings follow
Sec. 4 (10 points per wavelength: omega = 0.2 pi n at h = 1/n, a 16-cell quadratic layer,
beta = 0.5, three V(1,1) levels, coarsest GMRES(10), FGMRES(10), tolerance 1e-7).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass(frozen=True)
class Preset:
    name: str
    n: int                         # n x n grid, h = 1/n
    nrhs: int
    precond: str                   # "M_V", "M_JU", "M_VU", "encoder-solver M_VU"
    rhs_kind: str = "points"       # "points", or "points+gaussian" (half of each)
    train_pairs: int = 0           # Eq. 3.8-3.9 pairs of the medium (0: no network)
    train_epochs: int = 0
    train_lr: float = 1e-3
    train_batch: int = 16
    retrain_from: int = 0          # grid of the pretraining medium before mini-retraining (Sec. 3.5)
    tol: float = 1e-7
    notes: str = ""
    desc: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def omega(self) -> float:
        return synth.omega_for(self.n)

    def helmholtz_overrides(self) -> dict:
        """helm_desc fields for lib.Helmholtz(kappa2, **overrides)."""
        d = {"h": self.h, "omega": self.omega, "abc_width": 16, "levels": 3, "beta": 0.5}
        d.update(self.desc)
        return d

    def medium(self, problem: int = 0) -> np.ndarray:
        """kappa^2 (float32, n x n) of the seeded Gaussian-random-field medium."""
        return synth.grf_kappa2(self.n, self.n, synth.medium_seed(problem))

    def rhs(self, problem: int = 0) -> np.ndarray:
        """Right-hand sides (complex128, nrhs x n x n): point sources at least 16 cells from
        the edges, and for "points+gaussian" complex Gaussian noise in the second half."""
        npts = self.nrhs if self.rhs_kind == "points" else self.nrhs // 2
        pos = synth.source_positions(self.n, self.n, npts, synth.rhs_seed(problem), 16)
        b = synth.point_sources(self.n, self.n, pos, self.h)
        if self.rhs_kind == "points":
            return b
        return np.concatenate([b, synth.gaussian_rhs(self.n, self.n, self.nrhs - npts, 3000 + problem)])


PRESETS = {p.name: p for p in (
    Preset("plain_128", 128, 1, "M_V", notes="plain SL-FGMRES, the oracle's full-solve size"),
    Preset("general_256", 256, 8, "M_VU", train_pairs=1024, train_epochs=96,
           notes="the general network: 16 random media x 64 pairs (Sec. 3.4.1), solved on an unseen medium"),
    Preset("unet_256", 256, 8, "M_VU", train_pairs=300, train_epochs=20, train_lr=5e-4, retrain_from=256,
           notes="general network mini-retrained on the medium (the benchmark's 256^2 case)"),
    Preset("encoder_solver_512", 512, 32, "encoder-solver M_VU", rhs_kind="points+gaussian",
           train_pairs=512, train_epochs=40, notes="encoder on the medium once, solver network per call"),
    Preset("retrain_1024", 1024, 16, "M_VU", train_pairs=300, train_epochs=20, train_lr=5e-4, retrain_from=256,
           notes="network trained at 256^2, mini-retrained on the target medium"),
    Preset("retrain_2048", 2048, 16, "M_VU", train_pairs=300, train_epochs=20, train_lr=5e-4, train_batch=4,
           retrain_from=256, notes="the benchmark's headline case; training batch 4 by the network tensor limit "
                                   "(the solves run the network on chunks of 4 right-hand sides)"),
)}


def get(name: str) -> Preset:
    try:
        return PRESETS[name]
    except KeyError:
        raise ValueError(f"unknown preset {name!r}; known: {', '.join(PRESETS)}") from None
