"""Named workloads: event recipe, batch size, seeds and model shapes.

plain      1 event, 1 vertex, 20 tracks; embedding 3-32-32-4, k 16;
           interaction network hidden 32, 2 steps.
batch500   500 events, Poisson(5.3) vertices x Poisson(30) tracks; embedding
           3-128-128-128-8, k 32; hidden 128, 6 steps.
train64    64 events of the ``plain`` recipe; hidden 128, 6 steps (training).
pileup4x   1,000 events, Poisson(21) vertices x Poisson(30) tracks; hidden 128,
           8 steps.

Radii and logit cuts: the workload descriptions give radii 0.05 and 0.1,
meant for trained embeddings; with random weights they yield no edges.  The
values used here were produced by ``python -m oracle.calibrate`` (11.5
edges per hit on the calibration events; logit cut keeping the genuine-edge
fraction) and are recorded in oracle/calibration.json; pileup4x keeps the
batch500 radius (same embedding) with its own cut (its network has 8 steps).  The static
e4m3 activation scales (powers of two, 4 n_iters + 3 per network) come from
``python -m oracle.calibrate --fp8``: the amax of every tensor-core operand of
the exact forward over the first 40 (batch500) or 8 (pileup4x) calibration
events.  ``LITERAL_RADIUS``
keeps the described values for the degenerate-case tests.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

from .events import EventRecipe, make_batch
from .model import ModelConfig, make_weights

CALIB_SEED = 12345
CALIB_EVENTS = 200


@dataclass(frozen=True)
class Workload:
    name: str
    recipe: EventRecipe
    n_events: int
    base_seed: int
    model: ModelConfig

    def batch(self, n_events: int | None = None):
        return make_batch(self.recipe, self.n_events if n_events is None else n_events,
                          self.base_seed)

    def calibration(self):
        return make_batch(self.recipe, CALIB_EVENTS, CALIB_SEED)

    def weights(self, seed: int = 0, perturb: float = 0.0, calib=None):
        return make_weights(self.model, self.calibration() if calib is None else calib,
                            seed=seed, perturb=perturb)


PLAIN_RECIPE = EventRecipe(n_pv=1, tracks_per_pv=20)
PP_RECIPE = EventRecipe(n_pv=5.3, n_pv_poisson=True, tracks_per_pv=30, tracks_poisson=True)
PILEUP_RECIPE = EventRecipe(n_pv=21, n_pv_poisson=True, tracks_per_pv=30, tracks_poisson=True)

# log2 of the static e4m3 activation scales (python -m oracle.calibrate --fp8)
FP8_ACT_LOG2_BATCH500 = (-7, -6, -1, -6, -6, -6, -1, -7, -6, -6, 0, -6, -6, -6, 0, -7, -5, -6, 0, -7, -5, -6, 0, -6, -5, -7, -5)
FP8_ACT_LOG2_PILEUP4X = (-7, -6, 0, -6, -6, -6, 0, -7, -6, -6, 0, -6, -6, -6, 0, -7, -5, -7, 1, -6, -5, -6, 1, -7, -5, -7, 1, -7, -5, -7, 1, -7, -5, -7, -5)

BIG_MODEL = ModelConfig(emb_widths=(3, 128, 128, 128, 8), hidden=128, n_iters=6,
                        radius=1.14, k_max=32, threshold_logit=2.84772,
                        fp8_act_log2=FP8_ACT_LOG2_BATCH500)

LITERAL_RADIUS = {"plain": 0.05, "batch500": 0.1, "train64": 0.05, "pileup4x": 0.1}

WORKLOADS = {
    "plain": Workload("plain", PLAIN_RECIPE, 1, 1,
                      ModelConfig(emb_widths=(3, 32, 32, 4), hidden=32, n_iters=2,
                                  radius=1.5, k_max=16, threshold_logit=-1.37408)),
    "batch500": Workload("batch500", PP_RECIPE, 500, 1000, BIG_MODEL),
    "train64": Workload("train64", PLAIN_RECIPE, 64, 5000,
                        ModelConfig(emb_widths=(3, 32, 32, 4), hidden=128, n_iters=6,
                                    radius=1.5, k_max=16, threshold_logit=-0.717108)),
    "pileup4x": Workload("pileup4x", PILEUP_RECIPE, 1000, 9000,
                         replace(BIG_MODEL, n_iters=8, threshold_logit=0.422708,
                                 fp8_act_log2=FP8_ACT_LOG2_PILEUP4X)),
}
