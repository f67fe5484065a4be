"""Closed-form interconnect model of Sec. 3.3 ("Zero-Copy Mechanism and
Optimization"): TEST INFRASTRUCTURE ONLY.

The paper reasons about zero-copy reads with four plain formulas, restated
here in our own words:

* a link that can keep ``tags`` requests outstanding, each carrying
  ``req_bytes`` and taking ``rtt`` seconds to return, moves at most
  ``req_bytes * tags / rtt`` bytes per second (the paper's 8-bit PCIe tag
  field gives tags = 256);
* each transaction packet carries a fixed header, so the share of the wire
  spent on headers is ``header / (header + req_bytes)``;
* sustaining a bandwidth B with requests of ``req_bytes`` and round trip
  ``rtt`` needs ``ceil(B * rtt / req_bytes)`` requests in flight (Little's law);
* a DRAM whose smallest access is ``burst`` bytes serves a stream of
  ``req_bytes`` requests at ``peak * req_bytes / max(req_bytes, burst)``.

The paper quotes bandwidths in GB where it means 2^30 bytes (its 7.63 GB/s
is 8.192e9 B/s); ``GIB`` is used for that unit.
"""
from __future__ import annotations

import math

GIB = float(2 ** 30)


def tag_limited_bandwidth(req_bytes: float, rtt_s: float, tags: int = 256) -> float:
    """Upper bound on bytes/s from `tags` outstanding requests of `req_bytes`."""
    return req_bytes * tags / rtt_s


def header_overhead(req_bytes: float, header_bytes: float = 18.0) -> float:
    """Fraction of packet bytes spent on the header."""
    return header_bytes / (header_bytes + req_bytes)


def outstanding_needed(bandwidth_bps: float, rtt_s: float, req_bytes: float) -> int:
    """Requests that must be in flight to sustain `bandwidth_bps`."""
    return int(math.ceil(bandwidth_bps * rtt_s / req_bytes - 1e-9))


def dram_effective(peak_bps: float, req_bytes: float, burst_bytes: float = 64.0) -> float:
    """DRAM throughput seen by a stream of `req_bytes` requests."""
    return peak_bps * req_bytes / max(req_bytes, burst_bytes)


def aligned_start_probability(elem_bytes: int, line_bytes: int = 128) -> float:
    """Chance that a list starting at a uniformly random element index begins
    on a line boundary (Sec. 5.3.1)."""
    return elem_bytes / line_bytes
