"""GB300-native TPA: approximate Random Walk with Restart (arXiv 1708.02574).

Thin Python binding over the C ABI of ``libtpa.so`` (declared in
``include/tpa.h``).  Every step of the hot path -- CSR construction, the
cumulative power iteration (Algorithm 1), preprocessing (Algorithm 2) and the
online query (Algorithm 3) -- runs in the library's CUDA kernels; this module
only marshals arguments.  PyTorch provides device memory and the current
stream.  There is no CPU fallback: if the library cannot be loaded, every
call raises.
"""
from __future__ import annotations

from .tpa import (  # noqa: F401
    TpaError,
    Graph,
    Server,
    build_graph,
    cpi,
    cpi_exact,
    cpi_step_noalloc,
    edge_weights,
    loss_grad,
    set_adjoint_budget,
    set_adjoint_batch_width,
    get_adjoint_batch_width,
    set_edge_weights,
    sync,
    theta_grad,
    get_csr,
    get_stranger,
    graph_info,
    launch_count,
    library,
    profile_read,
    probe_gather,
    profile_reset,
    load_preprocessed,
    preprocess,
    query,
    query_sets,
    save_preprocessed,
    set_batch_width,
    set_output_group_width,
    get_output_group_width,
    set_cpi_batch_width,
    get_cpi_batch_width,
    set_push,
    set_pattern,
    seed_order,
    get_batch_width,
    set_variant,
    get_variant,
    variants,
)
from .autograd import TPALinkLoss  # noqa: F401,E402
