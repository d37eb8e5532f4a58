"""GB300-native FastPM particle-mesh loop (FlowPM, arXiv:2010.11847)."""
