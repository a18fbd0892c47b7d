"""FP64 CPU oracle of the multipole Poisson solve (test infrastructure only)."""
