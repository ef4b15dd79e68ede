"""Writes walkthrough_w4.json: an input whose split reproduces the example of Sec. 4.1.

The paper walks through one split of a 4-way interleaved stream (Sec. 4.1 and
its figure of the encoding/decoding of a split): the split sits on the word
that coder E4 wrote after symbol 16; the backward scan then meets E2 (after
symbol 14), E4 again (after symbol 12, ignored), E3 (after 11) and E1 (after 9).
The figure's symbols and distribution are not in the text, so this script
searches, with the oracle only, for a short input and a small parameter set
whose encoder produces exactly that pattern of renormalisations around one word.
The expected decoder behaviour is written in the test from the paper's prose,
not from this search.

Run from the repository root:  python tests/golden/make_walkthrough.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
import oracle  # noqa: E402

W, N_BITS, LGL, B = 4, 3, 4, 4
# paper's 1-based (coder, symbol) renormalisation records, oldest first
PAPER_EVENTS = [(1, 9), (3, 11), (4, 12), (2, 14), (4, 16)]


def search(seed=0, tries=200000):
    g = np.random.default_rng(seed)
    want = [(c - 1, s - 1) for c, s in PAPER_EVENTS]          # 0-based (lane, recorded index)
    for _ in range(tries):
        n_syms = int(g.integers(20, 29))
        sym = g.integers(0, 4, size=n_syms).astype(np.uint32)
        f = np.array([4, 2, 1, 1], dtype=np.uint32)             # sums to 2^3
        words, final, ev_sym, ev_y = oracle.encode(sym, f, N_BITS, W, LGL, B)
        rec = [(int(e % W), int(e - W)) for e in ev_sym]
        for q in range(len(rec)):
            if rec[q] != want[-1]:
                continue
            lo = q - len(want) + 1
            if lo < 0 or rec[lo:q + 1] != want:
                continue
            ok, idx, y, wp = oracle.scan(ev_sym, ev_y, q, W)
            if ok and list(idx) == [8, 13, 10, 15]:
                return sym, f, q
    raise RuntimeError("no input found")


def main():
    sym, f, q = search()
    out = {
        "citation": "Sec. 4.1 (Extending to Interleaved rANS) and Sec. 4.1.1-4.1.3 walkthrough",
        "note": "input found by tests/golden/make_walkthrough.py with the oracle encoder; "
                "expected decoder behaviour is taken from the paper's prose in the test",
        "W": W, "n": N_BITS, "lgL": LGL, "b": B,
        "f": [int(v) for v in f],
        "symbols": [int(v) for v in sym],
        "split_word": int(q),
        "paper_events_1based": PAPER_EVENTS,
    }
    path = os.path.join(os.path.dirname(__file__), "walkthrough_w4.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "split word", q, "N", len(sym))


if __name__ == "__main__":
    main()
