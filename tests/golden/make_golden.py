"""Writes tests/golden/exact_values.txt.  Calls only oracle.exact (brute-force
enumeration, Kaufman's finite-torus partition function, Onsager's energy and
Yang's magnetisation); nothing here touches the CUDA library.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

BETA_TC = 1.0 / 2.269


def main():
    lines = ["# Exact values for the 2D periodic Ising model (J=1, K=1, h=0).",
             "# Written by tests/golden/make_golden.py from oracle/exact.py.",
             "# kind L beta value"]
    for beta in (0.2, BETA_TC, 0.7):
        e, m, _, _ = exact.exact_means(4, beta)
        lines.append(f"enum_e_per_spin 4 {beta!r} {e!r}")
        lines.append(f"enum_absm_per_spin 4 {beta!r} {m!r}")
    for L, beta in ((16, BETA_TC), (8, 0.3), (8, 0.6), (42, 0.3), (42, 0.6), (42, BETA_TC)):
        lines.append(f"kaufman_e_per_spin {L} {beta!r} {exact.kaufman_energy(L, beta)!r}")
    for T in (1.0, 1.5, 2.0, 2.5, 3.0, 3.5):
        beta = 1.0 / T
        lines.append(f"onsager_e_per_spin inf {beta!r} {exact.onsager_energy(beta)!r}")
        lines.append(f"yang_m_per_spin inf {beta!r} {exact.yang_magnetization(beta)!r}")
    with open(os.path.join(HERE, "exact_values.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
