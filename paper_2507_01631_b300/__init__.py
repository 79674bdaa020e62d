"""B300-native (sm_103a) Snake-NeRF training step.

The product is the C-ABI library libsnk.so (include/snk.h, sources under
csrc/); `snk` is its ctypes binding and `trainer` allocates the device
tensors a step needs.  Build with `python -m paper_2507_01631_b300.build`.
"""
