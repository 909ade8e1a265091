"""FP64 CPU oracle -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference arm may import this package.  It shares no code with the CUDA path.
"""
from .isorank import (  # noqa: F401
    adjacency,
    adjacency_of,
    attribute_similarity,
    greedy_match,
    optimal_match,
    pair_score,
    propagate,
    restart_term,
    run_pairs,
    score_gradient,
    similarity,
)
from . import distances  # noqa: F401,E402  (interpolation + Table 1 distances)
from . import ward  # noqa: F401,E402  (Ward clustering of similarity profiles)
