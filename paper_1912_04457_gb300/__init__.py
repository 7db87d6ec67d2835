"""GB300-native Monte Carlo 2->2 collision term of the relativistic
Boltzmann equation with symmetrical sampling (arXiv:1912.04457).

The compute path is libbz.so (hand-written CUDA for sm_103a behind the C
ABI in include/bz.h); `bz` is its ctypes binding and `inputs` builds the
seeded synthetic initial states.
"""
