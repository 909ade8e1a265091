"""Seeded synthetic inputs (CFGs, attributes, pair lists) shared by the oracle
and the CUDA path.  No part of the similarity arithmetic lives here."""
from .cfg_grammar import CFG, loguniform_int, structured_cfg  # noqa: F401
from .configs import CONFIGS, Workload, all_pairs, config1, config2, config3, config4, config5  # noqa: F401
