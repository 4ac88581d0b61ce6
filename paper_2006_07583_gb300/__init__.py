"""GB300 (sm_103a) engine for the Peaceman-Rachford ADI step of the compact-FD and mimetic
acoustic schemes of arXiv 2006.07583.  The compute path is the C-ABI library libadi
(include/adi.h); ``adi`` is its thin ctypes binding."""
from .adi import (ADI_CFD, ADI_FP32, ADI_FP64, ADI_MFD, ADI_SOLVER_CHUNKED, ADI_SOLVER_FACTORED,
                  ADI_SOLVER_LINE, AdiError, Batch, Server, Sim, batch_poll, batch_submit, fixed_point, lib,
                  server_bytes, state_bytes)

__all__ = ["ADI_CFD", "ADI_MFD", "ADI_FP32", "ADI_FP64", "ADI_SOLVER_LINE", "ADI_SOLVER_CHUNKED", "ADI_SOLVER_FACTORED",
           "AdiError", "Sim", "Batch", "Server", "batch_submit", "batch_poll", "fixed_point", "lib", "state_bytes",
           "server_bytes"]
