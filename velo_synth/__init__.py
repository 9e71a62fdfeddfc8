"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Only input generation lives here (events, truth, weights, the blob format);
none of the track-finding arithmetic does.
"""
from .events import (N_PLANES, Z_PLANES, Batch, EventRecipe, compact_particle_ids, concat_events,
                     drop_noise, global_particle_ids,
                     make_batch, make_event, truth_edge_labels)
from .model import (ModelConfig, blob_layout, blob_size, make_triplet_weights, make_weights,
                    pack_blob, pack_triplet_blob, triplet_layout, unpack_blob)
from .presets import WORKLOADS, Workload

__all__ = ["N_PLANES", "Z_PLANES", "Batch", "EventRecipe", "compact_particle_ids", "concat_events",
           "drop_noise", "global_particle_ids",
           "make_batch", "make_event", "truth_edge_labels", "ModelConfig", "blob_layout",
           "blob_size", "make_weights", "pack_blob", "unpack_blob", "make_triplet_weights",
           "pack_triplet_blob", "triplet_layout", "WORKLOADS", "Workload"]
