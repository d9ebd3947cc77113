"""FP64 CPU oracle of SOGRAND and product-code turbo decoding.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.  Every function is documented in
``sogrand_oracle.c`` with the section of arXiv 2310.10737 it follows.

Parity pins (see tests/test_oracle_*.py): exhaustive 2^n enumeration on tiny
codes, partition counts, pattern distinctness and coverage, codeword
membership, the complement identity of the remaining mass, the closed form of
the L=1 corollary, the APP normalisation and, for product decoding, the
extrinsic exchange between half iterations (brute-force turbo chain with
exhaustive lists).
"""
from .oracle import (  # noqa: F401
    OracleCode, build, gldpc, gldpc_batch, lib, one_line_c, product, product_batch, product_trace, siso, siso_batch,
    trace,
)
