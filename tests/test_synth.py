"""The synthetic workloads stay the same graphs.

The generator's arrays are hashed (SHA-256 of every array's bytes and dtype);
a change to the generator that alters a single value of the tiny graph or of
the medium graph the bench times fails here.  The values were recorded from
the generator when its hot loops moved to multithreaded sorts and gathers,
which left every array unchanged (the large graph was checked the same way).
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2512_11606_gb300 import synth  # noqa: E402


def graph_hash(g) -> str:
    h = hashlib.sha256()
    for a in (g.e_u, g.e_v, g.e_w, g.ea_u, g.ea_a, g.ea_w):
        h.update(a.tobytes())
        h.update(str(a.dtype).encode())
    return h.hexdigest()[:16]


def test_tiny_and_medium_workloads_are_unchanged():
    assert graph_hash(synth.make_graph(**synth.TINY)) == "f01c13a790b50980"
    assert graph_hash(synth.make_graph(**synth.MEDIUM_BF16)) == "06e75dfd07365f53"


def test_bf16_round_matches_its_bit_definition():
    """Round to nearest bfloat16, ties to even, on random bit patterns and edge
    cases: (b + 0x7FFF + bit 16 of b) with the low 16 bits cleared, mod 2^32."""
    rng = np.random.default_rng(5)
    bits = np.concatenate([rng.integers(0, 2 ** 32, size=200_000, dtype=np.uint64).astype(np.uint32),
                           np.array([0, 0x7FFF, 0x8000, 0x18000, 0x3F808000, 0x3F818000, 0x7F7FFFFF,
                                     0xFFFF8000, 0xFFFFFFFF], np.uint32)])
    b = bits.astype(np.uint64)
    want = ((((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16) & 0xFFFFFFFF).astype(np.uint32)
    assert np.array_equal(synth.bf16_round(bits.view(np.float32)).view(np.uint32), want)
    # ties: 1 + 2^-8 (exactly halfway, even below) rounds down, 1 + 3 * 2^-8 rounds up
    assert synth.bf16_round(np.float32([1 + 2 ** -8, 1 + 3 * 2 ** -8])).tolist() == [1.0, 1 + 2 ** -6]
