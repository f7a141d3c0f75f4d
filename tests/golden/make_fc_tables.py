"""Writes the stored FC continuation tables in this folder.

Calls only ``oracle.fc_tables`` (mpmath, 60 digits).  The stored copies let
hosts without mpmath run the parity tests; ``tests/test_oracle_fc.py`` checks
that they equal a fresh build.

    python tests/golden/make_fc_tables.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fc_tables  # noqa: E402

if __name__ == "__main__":
    for d, C in [(5, 25), (5, 15), (7, 33)]:
        print(fc_tables.write_table(d, C, HERE))
