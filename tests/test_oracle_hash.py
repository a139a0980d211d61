"""Pin of the oracle's per-trajectory event hash.

The hash that parity compares (states aside) is FNV-1a 64 (Fowler, Noll, Vo)
over the little-endian bytes of each applied event's (uint32 rule, uint32
context slot), in event order, from the 64-bit offset basis. Here it is
recomputed from the oracle's own event logs with an FNV-1a written from its
definition. That implementation is first checked against published FNV-1a 64
test values.
"""
import numpy as np

import oracle
from paper_1010_2438_gb300 import workloads as W

FNV_OFFSET = 0xCBF29CE484222325
FNV_PRIME = 0x100000001B3


def fnv1a64(data: bytes, h: int = FNV_OFFSET) -> int:
    for b in data:
        h ^= b
        h = (h * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


def test_fnv1a64_published_values():
    # test values of the FNV-1a 64 reference suite (Noll's FNV page)
    assert fnv1a64(b"") == 0xCBF29CE484222325
    assert fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert fnv1a64(b"foobar") == 0x85944171F73967E8


def _check(batch, log_cap):
    o = oracle.simulate(batch, log_cap=log_cap, threads=4)
    assert o["events"].max() <= log_cap and o["events"].min() > 0
    for q in range(len(o["events"])):
        n = int(o["events"][q])
        data = b"".join(int(o["log_rule"][q, e]).to_bytes(4, "little") +
                        (int(o["log_slot"][q, e]) & 0xFFFFFFFF).to_bytes(4, "little") for e in range(n))
        assert fnv1a64(data) == int(o["hash"][q]), q


def test_flat_hash_is_fnv1a_of_the_event_log():
    b0 = W.flat8x12(R=8, G=10)
    _check(W.Batch(b0.model, b0.rates, b0.init, b0.grid * 0.02, b0.R, b0.seed), 4096)


def test_compartment_hash_is_fnv1a_of_the_event_log():
    c0 = W.cwc3x24(R=4, G=10)
    _check(W.Batch(c0.model, c0.rates, c0.init, c0.grid * 0.02, c0.R, c0.seed), 8192)
