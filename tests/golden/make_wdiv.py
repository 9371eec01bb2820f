"""Write tests/golden/wdiv.json: the head correction W^div of each input
configuration as computed by the CPU oracle (oracle.hamiltonian.head_correction,
Eqs. Wdiv, divergence_int, divergence_sum).  Calls only the oracle and the
input generator.  Run from the repository root:
    python tests/golden/make_wdiv.py si2 si4 lif4 mos2_331 mos2_331_uni si8 si12 lif10
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.hamiltonian import Inputs, head_correction  # noqa: E402
from synth import generate  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wdiv.json")


def main(names):
    out = json.load(open(PATH)) if os.path.exists(PATH) else {}
    for n in names:
        out[n] = head_correction(Inputs(generate(n)))
        print(n, repr(out[n]), flush=True)
    json.dump(out, open(PATH, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
