"""GB300 (sm_103a) implementation of the GOSH per-level graph-embedding step
(arxiv 2110.10049) behind the C ABI of include/gosh.h.

The compute lives in libgosh.so (csrc/*.cu); ``gosh`` is its ctypes binding.
"""
from . import gosh  # noqa: F401
from .gosh import (GoshError, Csr, Hierarchy, default_params, to_device_csr, gosh_validate_csr,  # noqa: F401
                   gosh_coarsen, gosh_init_embedding, gosh_train_level, gosh_project, gosh_embed,
                   gosh_pair_scores, gosh_link_auc, stats_dict)
