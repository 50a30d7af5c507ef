"""FP64 CPU oracle (test infrastructure only; see ns_oracle)."""
