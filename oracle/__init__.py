"""FP64 CPU oracle for the Gaussian Photon Field hit-point radiance query.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package. The product path (the CUDA library
and its Python binding) never imports, links or executes anything here, and
this package imports nothing from the product.

What it computes (paper arxiv 2512.12459):
  * forward radiance at hit points: Eq. (G_i) of Sec. 4.1, the aggregation
    L_GPF = sum_i w_i Phi_i with w_i = exp(-1/2 d^T Lambda_i d) psi(|d|) of
    Sec. 4.2 (Radiance Query and Aggregation), the soft falloff psi and the
    soft normalisation max(sum w, eps) of the query listing of Algorithm S3
    (Sec. A.2), the BSDF modulation of Sec. 4.2 read as a per-hit albedo and
    a hemisphere gate;
  * the analytic gradient of that output with respect to every Gaussian
    parameter (Sec. 4.2, Differentiable Accumulation), by the chain rule;
  * the MSE loss of Sec. 4.3 and its gradient;
  * the Adam update of Sec. A.2 (lr 5e-4);
  * the paper's hybrid neighbourhood, ball(r) or the k_min nearest means
    (Sec. 4.2, Neighborhood Search; Algorithm S3), and its gradient with the
    selection held fixed;
  * the per-view photon density estimate the field replaces (Sec. 3.2,
    Eq. kde; the gather of Algorithm S1), a disk kernel over photons.

Everything is a brute-force sum over all Gaussians in float64; the inputs are
the float32 values the GPU path receives, widened exactly.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, invariants, finite differences, library routines).
"""

from .gpf_oracle import (  # noqa: F401
    GPF_SUM,
    GPF_NORMALIZED,
    quat_to_rotmat,
    falloff_psi,
    radiance_fwd,
    radiance_bwd,
    disk_kde,
    hybrid_fwd,
    hybrid_bwd,
    mse_loss,
    mse_loss_grad,
    adam_step,
)
