"""FP64 CPU oracle of the three-phase colour-gradient LBM step (test infrastructure only)."""
