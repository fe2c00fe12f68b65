"""GB300-native exact hyper-triangle counting (Yin et al., PVLDB 18(3), 2024).

The computation runs in ``libhg.so`` (hand-written sm_103a CUDA kernels behind
the C ABI of ``include/hg.h``); ``hg`` is its ctypes binding with the same names.
Importing this package loads the library and fails if it is not built.
"""
from . import hg  # noqa: F401  (fails loudly when libhg.so is missing)
from .hg import (  # noqa: F401
    Graph, HgError, hg_build_wedges, hg_enumerate_pattern, hg_close_stats_get, hg_clustering_coeff, hg_count_patterns, hg_free,
    hg_kernel_launches, hg_kernel_times, hg_load_csr, hg_pattern_table, hg_canonical_masks,
    hg_mask_histogram, hg_count_owned, hg_out_degrees, hg_batch_mask_histogram, hg_autotune, hg_batch_autotune, hg_sample_estimate, hg_sample_estimate_adv, hg_sample_work_get, hg_set_allocator,
    hg_set_timing, hg_status_str, hg_wait_flag,
    use_default_allocator, use_torch_allocator,
    Batch, concat_members, hg_batch_build_wedges, hg_batch_clustering_coeff, hg_batch_count_patterns,
    hg_batch_free, hg_batch_waves, hg_load_batch, hg_load_batch_members,
    Server, HG_Q_COUNTS, HG_Q_CLUSTERING, HG_Q_ESTIMATE,
)


def count(num_vertices, edge_ptr, edge_vtx, stream=None):
    """Convenience: load, build, count and free; returns (counts uint64[21], wedge stats)."""
    g = hg_load_csr(num_vertices, len(edge_ptr) - 1, edge_ptr, edge_vtx, stream)
    try:
        stats = hg_build_wedges(g)
        counts = hg_count_patterns(g)
    finally:
        hg_free(g)
    return counts, stats
