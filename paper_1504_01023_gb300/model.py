"""The execution-time model of Sec. 4.5: a lower bound on the time per element,
the longer of the time to move the element's global data at a measured memory
bandwidth and the time to perform its operations at a measured arithmetic rate.

    t = max(bytes / bandwidth, operations / rate)

The paper states it in double-precision words (8 bytes) against STREAM bandwidth
and DGEMM throughput (Table 6 from Tables 4 and 5). The same bound, with this
library's algorithmic bytes and the measured GB300 copy bandwidth, is the
roofline that the benchmark reports."""
from __future__ import annotations


def time_bound_ns(bytes_per_element: float, ops_per_element: float, bandwidth_gbs: float,
                  rate_gflops: float) -> float:
    """Lower bound on the time per element in nanoseconds (GB/s and GFlop/s give
    bytes and operations per nanosecond)."""
    t_mem = bytes_per_element / bandwidth_gbs
    t_ops = ops_per_element / rate_gflops if rate_gflops > 0 else 0.0
    return max(t_mem, t_ops)


def paper_time_bound_ns(words: int, ops: int, stream_gbs: float, dgemm_tflops: float) -> float:
    """Table 6's estimate: `words` double-precision global accesses (Table 4) at the
    STREAM bandwidth, `ops` operations at the DGEMM rate (Table 5)."""
    return time_bound_ns(8.0 * words, ops, stream_gbs, dgemm_tflops * 1000.0)


def arithmetic_intensity(ops: int, words: int) -> float:
    """Operations per global double-precision word (Table 4)."""
    return ops / words
