"""FP64 CPU oracle of the ordering ICA. Test infrastructure only: used by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference legs, never by the library."""
from .ordering_ica import *  # noqa: F401,F403
