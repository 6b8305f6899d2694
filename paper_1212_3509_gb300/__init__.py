"""GB300-native demagnetizing operator as a sum of Kronecker products (arXiv 1212.3509).

The compute lives in ``lib/libdemag.so`` (CUDA, sm_103a) behind the C ABI of
``include/demag.h``; this package is a thin ctypes binding with the same
function names, plus a ``torch.autograd.Function`` for the demag energy.

There is no CPU fallback: importing the package requires the built library
(``paper_1212_3509_gb300.build.build()``), and every call needs a CUDA GPU.
"""
from ._abi import (  # noqa: F401
    DemagError,
    Graph,
    Plan,
    PRECISIONS,
    LIB_PATH,
    demag_apply_adjoint,
    demag_apply_cp,
    demag_apply_cp_batched,
    demag_apply_full,
    demag_build_factors_nonuniform,
    demag_compress_kernel,
    demag_compressed_ranks,
    demag_copy_compressed,
    demag_apply_tucker_compressed,
    demag_recompress_tucker,
    demag_round_tt,
    demag_apply_full_fft,
    demag_stray_field_fft,
    demag_energy_field_fft,
    demag_apply_full_batched,
    demag_apply_tt,
    demag_apply_tt_batched,
    demag_apply_tucker,
    demag_apply_tucker_batched,
    demag_autotune,
    demag_autotune_count,
    demag_autotune_entry,
    demag_build_factors,
    demag_copy_generators,
    demag_copy_nodes,
    demag_copy_symbols,
    demag_energy,
    demag_generators_size,
    demag_graph_create_batched,
    demag_graph_destroy,
    demag_graph_kernel_count,
    demag_graph_launch,
    demag_last_error,
    demag_num_terms,
    demag_plan_destroy,
    demag_reserve_workspace,
    demag_stray_field,
    demag_stray_field_exact,
    demag_symbols_size,
    demag_sync_status,
    demag_launch_count,
    demag_profile,
    demag_profile_count,
    demag_profile_launch,
    demag_profile_read,
    FAMILIES,
)
from .autograd import DemagEnergy, demag_energy_fn  # noqa: F401
