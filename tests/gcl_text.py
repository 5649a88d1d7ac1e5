"""Parse GCL text as the paper prints it ("CONST 0.5; LOAD b:1; ADD;") into wire tokens.

The paper's DIV, LN and SQRT are unprotected (Table 3); they map to PDIV, PLOG and PSQRT,
which agree with them wherever the test data keeps |divisor| > 1e-3, |log argument| > 1e-3
and the square-root argument non-negative.
"""
from __future__ import annotations

import os

from paper_2607_06731_gb300 import synth as S

_WORDS = {"ADD": S.ADD, "SUB": S.SUB, "MUL": S.MUL, "DIV": S.PDIV, "SIN": S.SIN,
          "COS": S.COS, "EXP": S.EXP, "LN": S.PLOG, "SQRT": S.PSQRT, "SQUARE": S.SQUARE,
          "DUP": S.DUP, "SWAP": S.SWAP, "DEL": S.DEL}

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse(text: str):
    toks = []
    for part in text.split(";"):
        part = part.strip()
        if not part:
            continue
        w = part.split()
        if w[0] == "CONST":
            toks.append((S.CONST, float(w[1])))
        elif w[0] == "LOAD":
            toks.append((S.LOAD0 + int(w[1].split(":")[1]), 0.0))
        else:
            toks.append((_WORDS[w[0]], 0.0))
    return toks


def paper_genomes():
    out = {}
    with open(os.path.join(GOLDEN, "paper_genomes.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, n, text = (s.strip() for s in line.split("|", 2))
            out[name] = (int(n), parse(text))
    return out
