"""B300-native stencil library for the hot path of arXiv 2310.01882.

The compute path is the CUDA C-ABI library built from csrc/ (libstencil.so).
`paper_2310_01882_b300.stencil` is the thin Python binding; importing this
package does not load the library, calling the binding does (and fails
loudly if it has not been built).
"""
__all__ = ["inputs"]
