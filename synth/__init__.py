"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This package draws random numbers and nothing else: it holds none of the blocked linear method's
arithmetic.  `synth.workload` builds host (numpy) arrays; `synth.device` fills device buffers with
the same draws through a small CUDA library of its own (libblmsynth.so).
"""
from .workload import (Workload, Model, workload, make_model, chunk, samples, equal_blocks,
                       uneven_blocks, batch_workloads)
