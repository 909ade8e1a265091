"""GB300-native CFG similarity for GPU-kernel subgraph matching.

The C ABI (include/cfsim.h, libcfsim.so) holds the whole hot path; this
package is its Python binding.  ``build.build()`` compiles the library for
sm_103a in-tree.
"""
from ._binding import CF_NORM_FROB, CF_NORM_NONE, CfsimError, lib  # noqa: F401


def __getattr__(name):
    # the torch-facing API is imported lazily so that the build step and the
    # CPU-only ABI checks do not need a CUDA device
    if name in ("Pack", "Workspace", "Result", "similarity", "match", "topk", "out_offsets", "ws_size",
                "similarity_backward", "CFSimilarity", "Graph", "probe", "autotune", "tune_info", "distances", "score_matrix", "ward"):
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
