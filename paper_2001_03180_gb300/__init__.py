"""GB300-native (sm_103a) FP64 implementation of the MSTAR hot path: one GBS extrapolation
step of the algorithmically regularised integrator with minimum-spanning-tree coordinates."""
