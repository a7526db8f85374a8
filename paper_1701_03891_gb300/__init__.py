"""DeepInverse (Mousavi & Baraniuk, arXiv 1701.03891) hot path for GB300 (sm_103a).

The compute path is ``libdeepinv.so`` (hand-written CUDA behind a C ABI, see
``include/deepinv.h``); ``deepinv`` is its thin Python binding.  Importing the
package does not load the library; the first call through the binding does,
and raises if the library is missing.
"""
__all__ = ["synth", "deepinv", "evaluate"]
