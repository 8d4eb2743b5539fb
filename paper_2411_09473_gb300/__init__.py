"""GB300 (sm_103a) IMM hot path: RRR-set sampling (IC reverse BFS, LT reverse
walk) and greedy max-coverage seed selection, as hand-written CUDA behind the
C ABI in include/imm.h (EfficientIMM, arXiv 2411.09473).

``paper_2411_09473_gb300.imm`` is the ctypes binding; it loads the in-tree
``_lib/libimm_gb300.so`` and fails loudly when that library is missing.
"""
from . import imm  # noqa: F401
from .imm import (IMM_IC, IMM_LT, ImmError, imm_create, imm_destroy, imm_get_counts,  # noqa: F401
                  imm_get_set, imm_get_sets, imm_last_error, imm_load_graph, imm_load_graph_device,
                  imm_reset_sets, imm_run, imm_sample, imm_select, imm_set_arena_limit, imm_stream_size)
