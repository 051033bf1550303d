"""Algorithmic HBM bytes of one direction-optimizing search, from its per-level records.

The records are the device counters the search itself returns (direction,
frontier size n_f and degree sum m_f, vertices found, bottom-up searchers and
their serial early-exit examination count).  The byte model charges what the
algorithm must move, independent of how the kernels move it.  With
W = ceil(n/8) bytes (one bitmap over all vertices) and `out` = 4 bytes per
requested output array (parent, level):

  init              out*n (fill) + W (completed bitmap)
  top-down level    16*n_f (two row offsets per frontier vertex) + 4*m_f (column ids)
                    + probe*m_f + (out + 4)*n_next (outputs + next-queue entry)
  bottom-up level   16*scanned + 4*examined + 3*W (read completed, write next,
                    update completed) + probe*examined + out*n_next
  queue -> bitmap   4*n_f + W      (before a bottom-up level that follows top-down)
  bitmap -> queue   W + 4*n_f      (before a top-down level that follows bottom-up)

probe = 0 bytes while a bitmap of n bits fits in a quarter of L2 (the
visited/frontier membership tests then stay on chip), else 4 bytes.
"""
from __future__ import annotations

L2_BYTES = 126 * 1024 * 1024


def search_bytes(n: int, records, want_parent: bool = True, want_level: bool = True) -> int:
    """records: rows (dir, nf, mf, nnext, mnext, scanned, examined[, t_ns]), one per level."""
    W = (n + 7) // 8
    out = 4 * (int(want_parent) + int(want_level))
    probe = 0 if W <= L2_BYTES // 4 else 4
    total = out * n + W
    prev = 0
    for r in records:
        d, nf, mf, nnext, _mnext, scanned, examined = (int(x) for x in r[:7])
        if d == 1 and prev == 0:
            total += 4 * nf + W
        elif d == 0 and prev == 1:
            total += W + 4 * nf
        if d == 0:
            total += 16 * nf + 4 * mf + probe * mf + (out + 4) * nnext
        else:
            total += 16 * scanned + 4 * examined + 3 * W + probe * examined + out * nnext
        prev = d
    return total
