"""FP64 CPU oracle (test infrastructure only; see coot_oracle)."""
