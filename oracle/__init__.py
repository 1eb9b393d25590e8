"""FP64 CPU oracle of the mechanical-interaction iteration (test infrastructure only)."""
