"""Plan autotuning (mf_autotune in the C library) with the tuned-plan cache of this package.

The tuner itself is native (csrc/autotune.cpp); this module only names the
default cache file, a JSON Lines file with one tuned plan per (device,
problem shape) key, and forwards the call.
"""
from __future__ import annotations

import os
from typing import Optional

from . import mfsolve as B

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_plans.jsonl")


def tune(analysis: "B.Analysis", values, b, base: Optional["B.mf_options"] = None, reps: int = 3,
         cache_path: Optional[str] = DEFAULT_CACHE, stream=None):
    """Tuned options for this analysis and its info dict (from the cache when it holds the key)."""
    return B.autotune(analysis, values, b, base=base, reps=reps, cache_path=cache_path, stream=stream)
