"""GB300 (sm_103a) implementation of the data-parallel E-step of ProSper's
truncated-posterior EM (arXiv 1908.06843) for BSC, TSC, DSC, MCA, MMCA and GSC.

The computation lives in hand-written CUDA kernels behind the C ABI of
``include/prosper.h`` (``_build/libprosper.so``); ``binding`` is a ctypes
wrapper around it and ``synth`` draws the seeded synthetic workloads.
"""
from . import binding, synth  # noqa: F401
from .binding import (BSC, MCA, GSC, TSC, DSC, MMCA, FP32, BF16_RESCORE, Context,  # noqa: F401
                      Params, ProsperError, load)
from .api import (BSC_ET, DSC_ET, EM, GSC_ET, MCA_ET, MMCA_ET, TSC_ET, LinearAnnealing,  # noqa: F401,E402
                  load_params, save_params)
