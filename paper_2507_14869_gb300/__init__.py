"""GB300-native lazy Probabilistic Cellular Automaton sampler for Bayesian
image denoising (arXiv 2507.14869).

The computation lives in ``libpcaden.so`` (hand-written CUDA for sm_103a,
C ABI declared in ``include/pcaden.h``).  This package is the thin ctypes
binding with the same entry-point names, plus the build step.
"""
from ._capi import (  # noqa: F401
    NOISE_FLIP, NOISE_GAUSS, NOISE_NONE, PAIR_POTTS, PAIR_TRUNC_LINEAR, SAMPLER_GIBBS_CB, SAMPLER_PCA,
    Chain, PcadError, PcadModel, as_model, lib, library_path,
    pcad_chain_create, pcad_chain_create_dev, pcad_chain_destroy, pcad_chain_export,
    pcad_chain_import, pcad_chain_metrics, pcad_chain_read_mean, pcad_chain_read_sample,
    pcad_chain_read_sample_dev, pcad_chain_reset, pcad_chain_run, pcad_chain_set_blocking, pcad_chain_stats, pcad_chain_sweeps,
    pcad_chain_set_kernel, pcad_chain_set_wait_limit, pcad_chain_inject_stall, PCAD_KERNEL_AUTO,
    pcad_chain_set_row_offset, pcad_chain_write_rows_dev,
    pcad_bands_create, pcad_bands_run, pcad_bands_sync, pcad_bands_read_sample,
    pcad_bands_read_mean, pcad_bands_info, pcad_bands_destroy, PCAD_KERNEL_CUDA_CORE, PCAD_KERNEL_TENSOR, PCAD_KERNEL_WAVE,
    PCAD_KERNEL_SMALL, PCAD_KERNEL_RESIDENT, PCAD_KERNEL_WINDOW, PCAD_KERNEL_WINDOW_WAVE,
    PCAD_KERNEL_BINARY,
    pcad_chain_energy, pcad_chain_track_energy, pcad_chain_read_energies,
    pcad_chain_read_min_state, pcad_chain_kernel_in_use, pcad_chain_set_model, pcad_chain_run_schedule,
    pcad_batch_set_model,
    pcad_chain_sync, pcad_chain_write_sample, pcad_last_error, pcad_metrics, pcad_status_str,
    pcad_pca_run_noalloc, pcad_version, pcad_model_margins, N_MARGINS,
    PcadJob, pcad_batch_create, pcad_batch_destroy, pcad_batch_info, pcad_batch_read_mean,
    pcad_batch_read_sample, pcad_batch_reset, pcad_batch_run, pcad_batch_sync,
    pcad_batch_set_tiling, pcad_batch_slice,
    pcad_server_create, pcad_server_destroy, pcad_server_info, pcad_server_poll,
    pcad_server_step, pcad_server_submit, pcad_server_set_limits, pcad_server_set_policy,
    SERVE_FIFO, SERVE_SRPT,
)
