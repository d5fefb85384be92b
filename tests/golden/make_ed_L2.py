"""Writes ed_L2.json: Trotterised exact-diagonalisation averages of the 8-site
(L=2) honeycomb Hubbard cluster, computed by the CPU oracle only (oracle/ed.py).
The GPU Monte Carlo chain must reproduce them within its statistical error,
because the HS sum is exact for the Trotterised density matrix at any dtau."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.lattice import Honeycomb  # noqa: E402
from oracle import ed  # noqa: E402

CASES = [dict(L=2, U=4.0, beta=1.0, dtau=0.125), dict(L=2, U=3.73, beta=2.0, dtau=0.125)]


def main():
    out = []
    for c in CASES:
        lat = Honeycomb(c["L"])
        M = int(round(c["beta"] / c["dtau"]))
        r = ed.trotter_averages(lat, lat.hopping_matrix(), c["U"], c["dtau"], M)
        out.append(dict(c, M=M, double_occ=r["double_occ"], energy=r["energy"], ekin=r["ekin"],
                        Czz=r["Czz"].tolist()))
    with open(os.path.join(HERE, "ed_L2.json"), "w") as f:
        json.dump({"source": "oracle/ed.py trotter_averages (tests/golden/make_ed_L2.py)", "cases": out}, f, indent=1)


if __name__ == "__main__":
    main()
