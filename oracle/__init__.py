"""FP64 CPU oracle for the twisted-mass Wilson hot path (test infrastructure only)."""
