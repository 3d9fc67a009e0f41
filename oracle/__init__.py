"""FP64 CPU oracle for RU-QLP (test infrastructure only; never on the product path)."""
from .ruqlp_oracle import (  # noqa: F401
    householder_qr, orth, jacobi_svd, apply_A, apply_At, ruqlp, ruqlp_paper,
    residual_fro, residual_fro_small, spectral_norm, principal_sines,
)
