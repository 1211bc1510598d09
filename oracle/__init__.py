"""FP64 CPU oracle of the well-balanced phase-field LBM (test infrastructure only)."""
