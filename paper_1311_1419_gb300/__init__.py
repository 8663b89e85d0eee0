"""GB300 (sm_103a) library for the multiple-residual block-CS video codec hot path."""
