"""FP64 CPU oracle for the PANDA message-passing iteration.

Test infrastructure only: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product path.
"""
