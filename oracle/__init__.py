"""CPU oracle for the UPIR region runtime.  Test infrastructure only: imported by
the tests, the smoke check and the benchmark's CPU baseline, never by the
library."""
