"""GB300-native streaming RX hyperspectral anomaly detection (hsad).

The compute path is the CUDA library ``libhsad.so`` (sources in ``csrc/``, C ABI in
``include/hsad.h``); :mod:`.hsad` is its ctypes binding. Build it with
``python -m paper_2602_13509_gb300.build``.
"""
from .hsad import *  # noqa: F401,F403
from .hsad import Detector, HsadError, header_functions, library, make_config  # noqa: F401
