"""GB300-native ADMM for the decomposed linearized (LinDist3Flow) OPF."""
