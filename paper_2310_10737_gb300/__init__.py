"""GB300-native SOGRAND (soft-output GRAND) and product-code turbo decoding.

Public entry points (same names as the C ABI in include/sogrand.h):

* :class:`Code` / :func:`sogrand_code_create` -- a component code from H;
* :func:`sogrand_decode` -- SISO decoding of many independent words;
* :func:`product_decode` -- block turbo decoding of product codes;
* :func:`product_decode_mixed` -- frames of several codes (uneven n) in one launch;
* :func:`gldpc_decode` -- QC-GLDPC codes on a component code (rows and wrapped diagonals);
* :class:`Server` -- continuous-batching decode service (requests admitted as slots free up);
* :func:`sogrand_trace_patterns` -- the device's canonical query order (test hook);
* :func:`sogrand_release_cached` -- hand the decoders' pooled scratch back to the device;
* :func:`sogrand_int_peak` -- the measured integer-pipe rate (the roofline's denominator);
* :func:`sogrand_set_wait_limits` -- bounds of the decoders' device-side waits;
* :mod:`calibration` -- predicted vs empirical list-BLER and BER (SOGRAND and Forney's approximation).

All compute runs in hand-written CUDA kernels for sm_103a (libsogrand.so);
PyTorch only provides device memory and streams.
"""
from ._lib import (  # noqa: F401
    Code, FrameGroup, LIB_PATH, ProductStats, Server, SograndError, load, product_decode, product_decode_host,
    product_decode_mixed, sogrand_code_create, gldpc_decode,
    sogrand_decode, sogrand_int_peak, sogrand_release_cached, sogrand_set_wait_limits, sogrand_trace_patterns,
    strerror, unpack_bits, DEFAULT_LOCK_POLLS, DEFAULT_QUEUE_WAIT_US,
    unpack_words,
)
