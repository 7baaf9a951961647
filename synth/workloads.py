"""Workload recipes: the synthetic inputs and method parameters of each case.

Every workload is a calorimeter-fill batch shaped like the experiment's
(Sec. 3): 54 crystals (6 x 9) per calorimeter, 560,000 samples per 700 us fill
at 800 MSPS, 12-bit ADC values held in int16.  Recipes only name sizes,
generator settings and the method's parameters; they compute nothing.
"""
from __future__ import annotations

import dataclasses
import math

from . import fill_plan, make_config

NOMINAL_SAMPLES = 560_000
SEED_BASE = 1611_04959


@dataclasses.dataclass
class Workload:
    name: str
    n_fills: int
    n_calo: int
    n_samples: int
    threshold: int
    pre: int
    post: int
    decim: tuple
    synth: dict
    uneven: dict | None = None          # fill_plan arguments for uneven fills
    ped_samples: int = 100

    def config(self):
        return make_config(n_fills=self.n_fills, n_calo=self.n_calo, n_samples=self.n_samples, **self.synth)

    def params(self) -> dict:
        return dict(threshold=self.threshold, pre=self.pre, post=self.post, ped_samples=self.ped_samples,
                    decim=tuple(self.decim))

    def plan(self):
        """(fill_len int32[F] or None, rate float64[F] or None)."""
        if not self.uneven:
            return None, None
        u = self.uneven
        return fill_plan(self.synth["seed"] + 17, self.n_fills, u["len_lo"], u["len_hi"], u["rate_lo"],
                         u["rate_hi"])

    @property
    def raw_bytes(self) -> int:
        return self.n_fills * self.n_calo * 54 * self.n_samples * 2


def _synth(idx: int, **kw) -> dict:
    d = dict(seed=SEED_BASE + idx, noise_sigma=3.0, pulses_per_fill=1500.0)
    d.update(kw)
    return d


# 1 calorimeter x 1 fill: the case the oracle finishes in seconds.
PLAIN_1CALO = Workload("plain 1 calorimeter x 1 fill (54 x 560,000 int16)", 1, 1, NOMINAL_SAMPLES,
                       30, 8, 24, (32,), _synth(0))
# Full single fill: 24 calorimeters x 54 crystals x 560,000 samples (1.4515 GB).
PLAIN_FULL_FILL = Workload("plain full fill (24 x 54 x 560,000 int16)", 1, 24, NOMINAL_SAMPLES,
                           30, 8, 24, (32,), _synth(1))
# Batching: 16 uneven fills (80k..560k samples, rate x log-uniform[0.2, 5]).
BATCH_UNEVEN = Workload("batch 16 uneven fills x 24 calorimeters", 16, 24, NOMINAL_SAMPLES,
                        30, 8, 24, (32,), _synth(2),
                        uneven=dict(len_lo=80_000, len_hi=560_000, rate_lo=0.2, rate_hi=5.0))
# Serving: stream of full fills (the pool of device fills cycles).
SERVING = Workload("serving stream of 24-calorimeter fills", 1, 24, NOMINAL_SAMPLES,
                   30, 8, 24, (32,), _synth(3))
# Stress: 48 fills x 24 calorimeters, 10x pulse rate, T=15, post=64, D in {8, 32}.
STRESS = Workload("stress 48 fills x 24 calorimeters, 10x rate", 48, 24, NOMINAL_SAMPLES,
                  15, 8, 64, (8, 32), _synth(4, pulses_per_fill=15000.0))
# Sparse regime: per-crystal noise 3/sqrt(54) so the 54-crystal sum has sigma ~3 ADC.
SPARSE_FULL_FILL = Workload("sparse full fill (sum noise sigma 3)", 1, 24, NOMINAL_SAMPLES,
                            30, 8, 24, (32,), _synth(5, noise_sigma=3.0 / math.sqrt(54.0)))

WORKLOADS = [PLAIN_1CALO, PLAIN_FULL_FILL, BATCH_UNEVEN, SERVING, STRESS]


def scaled(w: Workload, n_fills: int | None = None, n_calo: int | None = None, n_samples: int | None = None,
           **synth_overrides) -> Workload:
    """Same recipe at a smaller size (tests)."""
    s = dict(w.synth)
    s.update(synth_overrides)
    return dataclasses.replace(w, n_fills=n_fills or w.n_fills, n_calo=n_calo or w.n_calo,
                               n_samples=n_samples or w.n_samples, synth=s)
