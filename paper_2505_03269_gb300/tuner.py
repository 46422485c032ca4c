"""Autotuning with a persistent cache.

The paper tunes the work per thread block / warp and the number of buffers
per GPU and shape with Kernel Tuner and ships a default table (Sec. IV-A,
Table III).  Here the library times its own kernel configurations on the
caller's data (tcbf_autotune) and this module keeps the winners in a JSON
file keyed by device, mode and shape, so a shape is tuned once per GPU.

  from paper_2505_03269_gb300 import tuner
  info = tuner.tune_or_load(plan, Wp, Xp, Y)     # sets plan's configuration
"""
from __future__ import annotations

import json
import os
import threading

DEFAULT_PATH = os.environ.get(
    "TCBF_TUNING_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "tcbf", "tuning.json"))
_lock = threading.Lock()


def device_name(device: int) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def cache_key(plan) -> str:
    # the flags select the configuration table (stacked sample planes have their own)
    return (f"{device_name(plan.device)}|mode={plan.mode}|flags={getattr(plan, 'flags', 0)}|"
            f"batch={plan.batch}|M={plan.M}|N={plan.N}|K={plan.K}|w_batches={plan.w_batches}")


def _read(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def lookup(plan, path: str = DEFAULT_PATH):
    """Cached entry for this plan's shape, or None."""
    with _lock:
        return _read(path).get(cache_key(plan))


def tune(plan, Wp, Xp, Y, reps: int = 3, path: str = DEFAULT_PATH, store: bool = True) -> dict:
    """Time all configurations on the given buffers, keep the fastest on the
    plan and (optionally) record it in the cache."""
    best, ms = plan.autotune(Wp, Xp, Y, reps=reps)
    entry = {"config": best, "name": plan.config_name(best),
             "ms": {plan.config_name(i): t for i, t in enumerate(ms) if t >= 0}}
    if store:
        with _lock:
            data = _read(path)
            data[cache_key(plan)] = entry
            os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
            tmp = f"{path}.tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, path)
    return entry


def tune_or_load(plan, Wp, Xp, Y, reps: int = 3, path: str = DEFAULT_PATH) -> dict:
    """Apply the cached configuration for this shape, tuning it first if the
    cache has none."""
    entry = lookup(plan, path)
    if entry is not None and 0 <= entry.get("config", -1) < plan.num_configs():
        plan.set_config(entry["config"])
        return dict(entry, cached=True)
    return dict(tune(plan, Wp, Xp, Y, reps, path), cached=False)
