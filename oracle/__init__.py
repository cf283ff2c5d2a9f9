"""FP64 CPU oracle of the PSR-NQS hot path (test infrastructure only)."""
