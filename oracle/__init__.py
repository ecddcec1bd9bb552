"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Imported only by tests/, __graft_entry__.smoke() and the CPU-baseline leg of
bench.py.  The product path (paper_2507_15464_gb300) never imports it.
Parity status of each part is listed in the module docstrings.
"""
from .core import (Oracle, nrmse, fwhm, theta_ls, theta_ls_freq, tidas_conv,  # noqa: F401
                   tidas_conv_adjoint, tidas_conv2d, tidas_conv2d_adjoint, reference_row,
                   tidas_conv_varying, tidas_conv_varying_adjoint)
