"""FP64 CPU oracle (test infrastructure only; see cs_oracle's header)."""
