"""GB300-native coarse-grid projection (CGP) Poisson path for incompressible MHD."""
