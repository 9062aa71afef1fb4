"""FP64 CPU oracle of the porous-media MRT lattice Boltzmann model.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU baseline leg of ``bench.py``; the product package never imports it.
"""
from .orc import Lattice, Oracle, Physical, build, derive, lib  # noqa: F401
