"""Runs the library's tile search (flowroi_autotune) and writes the table.

    python -m paper_2511_14419_gb300.autotune --sizes 2048x2048 \\
        --storage 32 --streams 16 --out paper_2511_14419_gb300/tiles/gb300_fp32.json

The search itself is native (include/flowroi.h, "tile shapes"); this module
only marshals the arguments and writes the JSON text it returns.  A table
is read at create through config.tile_table.
"""
from __future__ import annotations

import argparse
import sys

from . import flowroi as F


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sizes", default="2048x2048", help="comma-separated WxH frame sizes")
    ap.add_argument("--storage", type=int, default=32, choices=[32, 16])
    ap.add_argument("--wavelet", type=int, default=97, choices=[53, 97])
    ap.add_argument("--dwt-levels", type=int, default=5)
    ap.add_argument("--pyr-levels", type=int, default=5)
    ap.add_argument("--streams", type=int, default=16, help="streams per batch while timing")
    ap.add_argument("--steps", type=int, default=4, help="batches timed per candidate")
    ap.add_argument("--base", default=None, help="a table to merge the result into (its other entries are kept)")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    sizes = [tuple(int(v) for v in s.lower().split("x")) for s in a.sizes.split(",")]
    cfg = F.flowroi_default_config(precision=a.storage, wavelet=a.wavelet, dwt_levels=a.dwt_levels,
                                   pyr_levels=a.pyr_levels, max_batch_frames=max(a.streams, 1))
    text = F.flowroi_autotune(cfg, sizes, a.streams, a.steps)
    if a.base:
        import json
        with open(a.base) as f:
            base = json.load(f)
        new = json.loads(text)
        keys = lambda e: (e["param"], e.get("w"), e["storage"], e.get("level"), e.get("kernel"))
        merged = {keys(e): e for e in base.get("entries", [])}
        merged.update({keys(e): e for e in new["entries"]})
        new["entries"] = list(merged.values())
        text = json.dumps(new, indent=2) + "\n"
    err = F.flowroi_tiles_check(text)
    if err:
        print(f"autotune produced an invalid table: {err}", file=sys.stderr)
        return 1
    with open(a.out, "w") as f:
        f.write(text)
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
