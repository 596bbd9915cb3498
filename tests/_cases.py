"""Shared, cached small cases for the CPU oracle tests."""

from __future__ import annotations

import functools

from synth import make_ground_state


@functools.lru_cache(maxsize=None)
def ground_state(name: str, kernel_mask: int = 3, collinear: bool = False):
    return make_ground_state(name, kernel_mask=kernel_mask, collinear=collinear)


@functools.lru_cache(maxsize=None)
def liouvillian(name: str, kernel_mask: int = 3, collinear: bool = False):
    from oracle.liouvillian import Liouvillian
    return Liouvillian(ground_state(name, kernel_mask, collinear))


@functools.lru_cache(maxsize=None)
def particle_hole(name: str, kernel_mask: int = 3, collinear: bool = False):
    from _bruteforce import ParticleHole
    lv = liouvillian(name, kernel_mask, collinear)
    return ParticleHole(lv.gs, lv.fxc)
