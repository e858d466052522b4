"""GB300 (sm_103a) library for the THC second-order-exchange self-energy.

The compute lives in ``libthcsox.so`` (hand-written CUDA behind a C ABI, see
``include/thc_sox.h``); this package is its thin Python binding plus a
``torch.autograd.Function`` around Phi_SOX.  Importing it does not build
anything; ``paper_2412_18829_gb300.build.build()`` compiles the library.
"""
from ._binding import (  # noqa: F401
    EXPORTED,
    Handle,
    PRECISIONS,
    SoxError,
    lib,
    phi_sox,
    phi_sox_backward,
    phi_sox_batch,
    phi_sox_grad_G,
    problem,
    sosex_dynamic_sigma,
    sox_w_dynamic,
    sosex_static_sigma,
    sox_check_device,
    sox_set_v_range,
    sox_set_kernel_variant,
    sox_dyson,
    sox_green_tails,
    sox_iw_to_tau,
    sox_tau_to_iw,
    sox_find_mu,
    sox_density_matrix,
    sox_sigma_hf,
    sox_gm_energies,
    sox_mix_green,
    sox_pi0,
    sox_profile_enable,
    sox_profile_read,
    sox_reserve,
    sox_sigma,
    sox_sigma_batch,
    g3w2_static_sigma,
    sosex2_static_sigma,
    SigmaBatchPlan,
    sox_sigma_fp64_noalloc,
    sox_sigma_general,
    sox_tau_grid,
    sox_version,
    sox_w_static,
    thc_project_G,
)
from .autograd import PhiSOX  # noqa: F401
