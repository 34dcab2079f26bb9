"""Plain FP64 CPU oracle of the micro-macro KFVS step (test infrastructure only)."""
