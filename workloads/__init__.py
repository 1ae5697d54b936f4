"""Seeded synthetic IMDP inputs shaped like the benchmark models of arXiv
2401.04068 (Appendix B, the 35-model table).  This package builds inputs only;
it holds none of the value-iteration arithmetic, and both the oracle tests and
the CUDA path take their inputs from it."""
from .imdp_synth import (  # noqa: F401
    IMDPInput,
    banded_imdp,
    banded_batch,
    random_imdp,
    concat_block_diagonal,
    CONFIGS,
    make_config,
)
