"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package builds the *inputs* of SOGRAND decoding and nothing else:

* ``codes``   – parity-check / generator matrices of the even component codes
                (extended BCH / extended Hamming) and the product encoder;
* ``channel`` – counter-based seeded BPSK-over-AWGN channel LLRs;
* ``fading``  – block Rician fading with Gray QPSK and interleaving;
* ``gldpc``   – QC-GLDPC codes on a component code (rows and wrapped diagonals).

It holds none of the decoding arithmetic (no query order, no soft output), so
the oracle and the GPU path can both consume its outputs without sharing any
of the method's code.
"""
from .codes import LinearCode, ebch, shorten, CODE_SPECS  # noqa: F401
from .channel import awgn_frames, awgn_words, sigma2_for  # noqa: F401
from .fading import fading_frames  # noqa: F401
from .gldpc import QCGLDPC, gldpc_frames  # noqa: F401
