"""B300-native heterogeneity-aware N-way majority voter.

The voter of Sec. IV.D of Kicherer & Karl ("Heterogeneity-aware Fault Tolerance
using a Self-Organizing Runtime System"): R redundant task results are compared
element by element (bit-wise for integers, within a stated tolerance for floating
point), the presumable correct result is written out, per-replica mismatch counts
and first-mismatch indices are reported, and a CRC32C per 4 KiB block of the
voted buffer is produced.  All compute runs in hand-written sm_103a CUDA kernels
behind the C ABI declared in ``include/ftvote.h``; ``ftvote`` is the thin ctypes
binding with the same entry-point names.  Importing this package does not load
the CUDA library; ``paper_1405_2912_b300.ftvote`` does, and fails loudly if it is
missing.
"""
__all__ = ["ftvote", "synth"]
