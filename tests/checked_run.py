"""Run the checked_cases with the package as imported (meant for
GS_LIBRARY=checked in a process of its own) and store the outputs
(npz) and the refused-access counts (json).  Usage: checked_run.py OUT.npz
OUT.json"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402


def main():
    import torch

    import paper_2501_09398_gb300 as g
    from checked_cases import cases, heat

    assert g.gs_debug_checked_build(), "not the checked build"
    torch.cuda.set_stream(torch.cuda.Stream())
    arrays, refused = {}, {}
    for name, fn in cases():
        outs, ref, _ = fn(g)
        refused[name] = list(ref)
        for k, o in enumerate(outs):
            arrays[f"{name}#{k}"] = o
    # planted: P left out of the table -> its loads are refused (and skipped)
    _, ref, pspan = heat(g, 77, 45, 1, 3, 0, dict(kernel=4, rows=8), omit_p=True)
    refused["planted: P not registered"] = list(ref) + list(pspan)
    np.savez(sys.argv[1], **arrays)
    with open(sys.argv[2], "w") as f:
        json.dump(refused, f)


if __name__ == "__main__":
    main()
