"""GB300-native FFT-based quasi-periodic Green's functions (Zhang & Zhang, arXiv:1801.05977)."""
