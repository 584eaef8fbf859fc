"""GB300-native learned indexed nested loop join (RMI-INLJ).

Sabek and Kraska, "The Case for Learned In-Memory Joins": a two-level linear
Recursive Model Index is fitted over the sorted inner relation R, then every
outer key of S predicts a position, searches the model's error window and
emits all matching (r_idx, s_idx) pairs.  The computation runs in the CUDA
library `libljoin` (hand-written sm_103a kernels, C ABI in include/ljoin.h);
this package is its thin Python binding.  The library is loaded on first
use; there is no CPU fallback.
"""
from ._native import (LJ_FP32, LJ_FP64, BatchPlan, Index, LJoinError, Server, grmi_build,
                      grmi_drop, grmi_export, grmi_stats, join_batch, join_expand,
                      join_locate, lhash_build, lhash_build_rs, lhash_export_first, index_autotune,
                      join_batch_plan, join_count, join_count_noalloc, join_emit, join_host, lsj_join,
                      rmi_autotune, rmi_autotune_clear,
                      library_path, lj_get_option, lj_last_error, lj_profile_report,
                      lj_set_option,
                      lj_version, load, rmi_build, rmi_build_batch, rmi_export,
                      rmi_free, rmi_stats, rs_export, rs_export_table)

__all__ = ["LJ_FP32", "LJ_FP64", "BatchPlan", "Index", "LJoinError", "Server", "grmi_build",
           "grmi_drop", "grmi_export", "grmi_stats", "join_batch", "join_expand",
           "join_locate", "lhash_build", "lhash_build_rs", "lhash_export_first", "index_autotune",
           "join_batch_plan", "join_count", "join_count_noalloc", "join_emit", "join_host",
           "lsj_join",
           "rmi_autotune", "rmi_autotune_clear",
           "library_path", "lj_get_option", "lj_last_error", "lj_profile_report",
           "lj_set_option", "lj_version", "load", "rmi_build", "rmi_build_batch", "rmi_export",
           "rmi_free", "rmi_stats", "rs_export", "rs_export_table"]
