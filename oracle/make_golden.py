"""Regenerate the stored expected values that come from the oracle.

Writes tests/golden/group_constants.json: blackbody (1e5 K) group attributes
for the three bands and the single band of the paper's Sec. 6 tests,
computed with oracle.groups only.  Run:  python -m oracle.make_golden
"""
import json
import os

from oracle import groups

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "tests", "golden", "group_constants.json")


def main():
    res = {"_about": "written by oracle/make_golden.py from oracle/groups.py (Eqs. (csn_multi), "
                     "(egy_multi), (cse_multi) with the Verner fits, 1e5 K blackbody)"}
    for name, bands in (("three_band", groups.THREE_BANDS), ("one_band", groups.ONE_BAND)):
        a = groups.group_attributes(bands, 1e5)
        res[name] = {
            "bands_eV": [[lo, (hi if hi != float("inf") else "inf")] for lo, hi in bands],
            "sigN": a["sigN"].tolist(), "sigE": a["sigE"].tolist(),
            "egy_eV": (a["egy"] / groups.EV).tolist(),
            "photon_fraction": a["photon_fraction"].tolist(),
        }
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
