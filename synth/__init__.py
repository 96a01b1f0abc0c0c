"""Seeded synthetic workloads for the ordering-ICA hot path (inputs only)."""
from .generators import *  # noqa: F401,F403
