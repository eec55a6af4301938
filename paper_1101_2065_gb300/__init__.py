"""GB300-native GW screening pipeline (arXiv:1101.2065, Foerster, Koval,
Sanchez-Portal): chi0 -> W -> Sigma -> diagonal quasiparticle equation on one
GPU, behind the C ABI of libgw.so (include/gw.h).

The Python layer is a ctypes binding (``gw``) and the in-tree build
(``build``); all computation runs in the CUDA library.
"""
from . import build
from .gw import (GW_FP64, GW_MIXED, GW_OPT_FORMS_SIMT, GW_OPT_SYRK_SIMT, GW_OPT_GEMM_SIMT, GW_OPT_KK_TENSOR, GW_OPT_POLES_FP64, GW_OPT_BARRIER_POLLS, Context, GWError, Server, gw_build_chi0, gw_build_chi0_thr, gw_build_chi0_2w, gw_sigma_diag_2w, solve_two_window, gw_sigma_matrix, gw_sigma_matrix_copy, gw_dyson_dos, dos_peak, gw_mol_upload, gw_qp_solve,
                 gw_screen_W, gw_sigma_diag, gw_solve, gw_solve_host, load, solve)

__all__ = ["build", "GW_FP64", "GW_MIXED", "GW_OPT_FORMS_SIMT", "GW_OPT_SYRK_SIMT", "GW_OPT_GEMM_SIMT", "GW_OPT_KK_TENSOR", "GW_OPT_POLES_FP64", "GW_OPT_BARRIER_POLLS", "Context", "GWError", "Server", "gw_build_chi0", "gw_build_chi0_thr", "gw_build_chi0_2w", "gw_sigma_diag_2w", "solve_two_window", "gw_sigma_matrix", "gw_sigma_matrix_copy", "gw_dyson_dos", "dos_peak", "gw_mol_upload",
           "gw_qp_solve", "gw_screen_W", "gw_sigma_diag", "gw_solve", "gw_solve_host", "load", "solve"]
