"""GB300-native HOG face detection (pyramid, gradient histograms, 31-d
features, multi-filter correlation, threshold and NMS) behind a C ABI.

The compute path lives in ``csrc/`` (CUDA for sm_103a) and is reached through
``paper_2006_00816_gb300.hog`` (ctypes marshalling only).  Importing the
package itself loads nothing; ``hog`` loads ``libhog.so`` and fails loudly if
it is missing.
"""
__all__ = ["hog", "synth"]
