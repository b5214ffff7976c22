"""FP64 CPU oracle of the RTM-GD tracer -- test infrastructure only.

Only tests/, the smoke check and the CPU-baseline leg of bench.py import this
package; the CUDA product path never does.
"""
