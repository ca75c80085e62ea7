"""GB300-native solver for the variational-embedding SDP relaxation of Khoo & Lindsey
(arXiv:2106.02682): translation-invariant ADMM / projected dual ascent (Algorithm 6) on one
GPU behind the C ABI of include/ve.h.

`from paper_2106_02682_gb300 import ve` loads the compiled library (libve_gb300.so, built by
paper_2106_02682_gb300.build); there is no CPU fallback.
"""
__all__ = ["ve", "build"]
