"""GB300 (sm_103a) implementation of the hot path of ARC, the photon-conserving
adaptive ray tracer of Hartley & Ricotti (arXiv 1807.07094).

The compute path is libarc.so (CUDA kernels behind the C ABI in
include/arc.h); ``arc`` is its thin ctypes binding.
"""
from .arc import (Arc, ArcError, ArcGrid, ArcParams, arc_add_sources, arc_chem_update,  # noqa: F401
                  arc_clear_sources, arc_create, arc_destroy, arc_get_fields,
                  arc_get_record_count, arc_last_error, arc_set_fields, arc_set_records,
                  arc_set_tuning, arc_get_tuning, arc_autotune, arc_stats, arc_step, arc_trace,
                  device_view, load, make_params, arc_set_surrogate, MlpTrainer, arc_mlp_eval,
                  arc_mlp_features, arc_mlp_targets, load_surrogate, SURROGATE_FILE,
                  REC_DTYPE)
