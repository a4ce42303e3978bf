"""GB300-native (sm_103a) Parareal for the Cahn-Hilliard equation.

Linear and nonlinear Parareal methods of Garai & Mandal (arXiv 2304.14074): the fine
propagator over all time slices at once, the coarse sweep and the correction of Eq. 2.2,
implemented as hand-written CUDA behind the C ABI of ``include/ch_parareal.h``. This
package is the thin Python binding of that ABI.
"""
from ._lib import (CH_GTHETA_PARAMS, CH_MAX_ITERS, EXPORTED_SYMBOLS, SCHEMES, STATUS, VARIANTS, ChError, Config,
                   Ensemble, GTheta, Parareal, gtheta_flatten, gtheta_unflatten, load, propagate, sine_transform_2d,
                   theory_bound, wait_selftest)
from .metrics import append_jsonl, stats_records
from .build import LIB as LIBRARY_PATH
from .build import build

__all__ = ["CH_GTHETA_PARAMS", "CH_MAX_ITERS", "EXPORTED_SYMBOLS", "SCHEMES", "STATUS", "VARIANTS", "ChError",
           "Config", "Ensemble", "GTheta", "Parareal", "gtheta_flatten", "gtheta_unflatten", "load", "propagate",
           "sine_transform_2d", "theory_bound", "wait_selftest", "build", "LIBRARY_PATH", "stats_records",
           "append_jsonl"]
