"""FP64 CPU oracle of the PIC Monte Carlo time step (test infrastructure only)."""
