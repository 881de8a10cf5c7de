"""FP64 CPU oracle of the BOS forward model (test infrastructure only)."""
