"""FP64 CPU oracle for the ConKer hot path.  Test infrastructure only: the
tests, the smoke check and the bench's CPU-baseline leg use it; the library
never does."""
