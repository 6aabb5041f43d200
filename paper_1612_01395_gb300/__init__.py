"""GB300-native pipelined BiCGStab (Cools & Vanroose, arXiv:1612.01395)."""
