"""CPU oracle (test infrastructure only; never imported by the product path).

See rydberg.py for what it computes and the passages of arXiv 2510.09813 it
follows.
"""
from .rydberg import *  # noqa: F401,F403
