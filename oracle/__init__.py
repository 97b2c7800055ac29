"""FP64 CPU oracle of the monodomain IMEX step (test infrastructure only)."""
