"""Write rate_constants.json: the numbers of every rate-coefficient fit of
the paper's appendix "Interaction rate coefficients adopted in RamsesRT",
taken mechanically from the paper's LaTeX source (no hand transcription).

For each fit the numbers of its right-hand side are listed in the order in
which they are printed, as strings and as floats: "a \\times 10^{b}" is one
number (a * 10^b), "10^{b}" alone is 10^b, digit groups written with a thin
space ("157 \\ 809.1") are joined, and a minus sign written directly in
front of a number (as in e^{-157 809.1/T} or T^{-1.5}) belongs to it.  The
rate names are the LaTeX macros of the paper with their species subscript.

The test test_oracle_rate_constants.py reads the JSON; rerun this script
only to regenerate it:

    python tests/golden/extract_rate_constants.py <path of the paper's LaTeX source>
"""
import json
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def _join_groups(s):
    prev = None
    while prev != s:
        prev = s
        s = re.sub(r"(\d{1,3}) *\\ +(\d{3})(?!\d)", r"\1\2", s)
    return s


NUM = re.compile(r"(?<![\w.])10\^\{?(-?\d+)\}?|(?<![\w.])(-?\d+(?:\.\d+)?)(?:\s*\\times\s*10\^\{(-?\d+)\})?")


def numbers(rhs):
    rhs = _join_groups(rhs)
    out = []
    pos = 0
    while True:
        m = NUM.search(rhs, pos)
        if not m:
            break
        pos = m.end()
        if m.group(1) is not None:          # 10^{b} alone
            txt = "1e%s" % m.group(1)
        elif m.group(3) is not None:        # a \times 10^{b}
            txt = "%se%s" % (m.group(2), m.group(3))
        else:
            txt = m.group(2)
        out.append(txt)
    return out


def main(path):
    src = open(path).read()
    start = src.index(r"\section{Interaction rate coefficients adopted in RamsesRT}")
    end = src.index(r"\subsection{Cross sections}", start)
    sec = src[start:end]
    fits = {}
    for block in re.findall(r"\\begin\{align\*\}(.*?)\\end\{align\*\}", sec, flags=re.S):
        for eq in block.split(r"\\"):
            eq = " ".join(eq.split())
            if "&=" not in eq:
                continue
            lhs, rhs = eq.split("&=", 1)
            name = lhs.strip().replace(" ", "")
            # the printed equalities "= k_B T alpha = k_B T 3e-14 ..." keep their last form
            if "=" in rhs:
                rhs = rhs.split("=")[-1]
            rhs = rhs.replace("&", " ")
            nums = numbers(rhs)
            fits[name] = {"latex": rhs.strip(), "numbers": nums, "values": [float(v) for v in nums]}
    out = {"_about": "Numbers of the rate fits of the paper's appendix 'Interaction rate coefficients adopted "
                     "in RamsesRT' (Rosdahl et al. 2013), extracted mechanically from its LaTeX source by "
                     "extract_rate_constants.py, in printed order per fit.",
           "fits": fits}
    with open(os.path.join(HERE, "rate_constants.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return fits


if __name__ == "__main__":
    if len(sys.argv) != 2:
        raise SystemExit(__doc__)
    fits = main(sys.argv[1])
    for k, v in fits.items():
        print(k, v["numbers"])
