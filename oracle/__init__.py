"""Plain FP64 CPU oracle for global and streaming RX anomaly detection, and subsampled
kernel RX (``oracle.krx``).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package. The
library in ``paper_2602_13509_gb300`` never calls it and shares no code with it.

Every function is pinned by tests/test_oracle_*.py against brute force in
exact rational arithmetic, closed forms, exact invariants and library
routines (see each function's docstring for its pin).
"""
from .rx import (  # noqa: F401
    ABS,
    CUBE,
    EXCLUSIVE,
    INCLUSIVE,
    REL,
    NotPositiveDefinite,
    calibrate,
    cholesky_lower,
    encode_tx,
    forward_substitution,
    forget_weights,
    frontend,
    gain_correct,
    global_rx,
    rx_scores,
    sample_covariance,
    sample_mean,
    statistics_lines,
    stream_rx,
    stream_rx_line,
    threshold_mask,
)
from . import krx  # noqa: F401,E402
