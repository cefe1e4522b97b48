"""GB300-native hit-point radiance of a Gaussian Photon Field (arxiv 2512.12459).

The compute path is libgpf.so (CUDA, sm_103a; C ABI in include/gpf.h). This
package is its Python binding: PyTorch tensors for memory and streams,
ctypes for the calls. The library is loaded at the first call; every call
raises if libgpf.so has not been built (there is no fallback path)."""

from . import _abi
from ._abi import (GPF_FLAG_CAPACITY, GPF_FLAG_NONFINITE, GPF_FLAG_TIMEOUT, GPF_PEAK_EX2,
                   GPF_PEAK_FP32_FMA, GPFError, LIB_PATH, load)
from .api import (GPF_DISK_KDE, GPF_NB_BALL_KNN, GPF_NB_KSIGMA, GPF_NORMALIZED, GPF_SUM, PAPER_EPS, PAPER_LR, PAPER_R,
                  AdamState, Field, GridConfig, Index, Queries, gpf_adam_step, gpf_count_pairs,
                  gpf_launch_count, gpf_measure_alu_peak, gpf_mse_loss_grad,
                  gpf_mse_workspace, gpf_radiance_bwd, gpf_radiance_fwd, gpf_sort_pairs,
                  grid_for_bounds, photon_field)
from .autograd import GPFRadiance, gpf_radiance

__all__ = [
    "GPFError", "LIB_PATH", "load", "GPF_NORMALIZED", "GPF_SUM", "GPF_DISK_KDE", "PAPER_EPS",
    "GPF_NB_KSIGMA", "GPF_NB_BALL_KNN",
    "PAPER_LR", "photon_field",
    "PAPER_R", "AdamState", "Field", "GridConfig", "Index", "Queries", "gpf_adam_step",
    "gpf_mse_loss_grad", "gpf_radiance_bwd", "gpf_radiance_fwd", "grid_for_bounds",
    "gpf_count_pairs", "gpf_launch_count", "gpf_sort_pairs",
    "GPFRadiance", "gpf_radiance", "_abi", "gpf_measure_alu_peak", "gpf_mse_workspace",
    "GPF_FLAG_CAPACITY", "GPF_FLAG_TIMEOUT", "GPF_FLAG_NONFINITE", "GPF_PEAK_FP32_FMA",
    "GPF_PEAK_EX2",
]
