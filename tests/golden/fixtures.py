"""Readers for the text fixtures in this directory (no computation)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def read_kv(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(" ")
            out[key] = val.strip()
    return out


def ints(s: str) -> list:
    return [int(x) for x in s.split(",") if x != ""]


def fig3():
    kv = read_kv("fig3.txt")
    rows = {}
    for tok in kv["rows"].split():
        r, _, cs = tok.partition(":")
        rows[int(r)] = ints(cs)
    return {
        "rows": rows,
        "jc": ints(kv["dcsc_jc"]), "cp": ints(kv["dcsc_cp"]), "ir": ints(kv["dcsc_ir"]),
        "split": [(ints(kv["split0_jc"]), ints(kv["split0_cp"]), ints(kv["split0_ir"])),
                  (ints(kv["split1_jc"]), ints(kv["split1_cp"]), ints(kv["split1_ir"]))],
        "root": int(kv["root"]), "level": ints(kv["level"]), "parent": ints(kv["parent"]),
    }
