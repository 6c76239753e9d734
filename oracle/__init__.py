"""Plain FP64 CPU oracle of the lattice Boltzmann hot path (test infrastructure only)."""
