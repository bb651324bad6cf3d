"""CPU oracle for the checkerboard hard-particle MC sweep (test infrastructure only)."""
