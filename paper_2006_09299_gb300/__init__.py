"""GB300-native run-based black-and-white connected component analysis.

The compute path is the CUDA library built from csrc/ (libccl.so, sm_103a),
reached through the ctypes binding in ccl.py. Importing this package does not
load the library; `paper_2006_09299_gb300.ccl` does, and raises if it is
missing.
"""
