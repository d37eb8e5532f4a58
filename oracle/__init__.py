"""FP64 CPU oracle of the particle-mesh loop (test infrastructure only)."""
