"""Reference block-step scheduler (test infrastructure only: the tests, the package smoke
check and the benchmark's CPU legs may use it; the library never does).

It states the scheduling of hierarchical power-of-two block steps (Sec. 2: steps are
integer powers of 1/2; Sec. 3.3.1: the particles are kept in a list sorted by step, and
after each block step the active particles' new steps re-sort it) by its plain definition,
without the paper's boundary offsets:

  * every particle i has a level L_i (step 2^-L_i) and the time t_i of its last step; times
    are integers in ticks of 2^-tick_level;
  * the next block time is the smallest next time t_i + 2^-L_i over all particles, and the
    active particles are all those whose next time equals it (a brute-force search);
  * after the step, an active particle takes the level the integrator requests, under the
    block rule: the request is clamped to [level_min, level_max]; a larger step than twice
    the current one is cut to one doubling; a doubling is granted only when the block time
    is a multiple of the doubled step (else the level stays);
  * the list is the particles ordered by step, smallest first (level descending), ties in
    their previous list order (a stable sort of the whole list after every step).
"""
from __future__ import annotations

import numpy as np


class SortingList:
    def __init__(self, levels, level_min: int = 0, level_max: int = 40, tick_level: int = 48):
        levels = np.asarray(levels, dtype=np.int64)
        if levels.min() < level_min or levels.max() > level_max or level_max > tick_level:
            raise ValueError("levels outside [level_min, level_max] or level_max > tick_level")
        self.level = levels.copy()
        self.level_min, self.level_max, self.tick = level_min, level_max, tick_level
        self.t_last = np.zeros(levels.shape[0], np.int64)
        self.T = 0
        self.order = np.argsort(-self.level, kind="stable")
        self.n_active = 0

    def step_ticks(self, level):
        return np.left_shift(np.int64(1), self.tick - np.asarray(level, np.int64))

    def next(self):
        """Advance to the next block time; returns (T_new in ticks, sorted active indices)."""
        t_next = self.t_last + self.step_ticks(self.level)
        self.T_new = int(t_next.min())
        active = np.nonzero(t_next == self.T_new)[0]
        self.n_active = active.size
        return self.T_new, active

    def update(self, want):
        """Apply the requested levels of the active particles, given in list order (the
        first n_active entries of the list), then re-sort the list."""
        act = self.order[:self.n_active]
        assert np.all(self.t_last[act] + self.step_ticks(self.level[act]) == self.T_new)
        L = self.level[act]
        w = np.clip(np.asarray(want, np.int64), self.level_min, self.level_max)
        w = np.maximum(w, L - 1)
        doubling = w == L - 1
        commensurate = self.T_new % self.step_ticks(np.maximum(L - 1, 0)) == 0
        w = np.where(doubling & ~commensurate, L, w)
        self.level[act] = w
        self.t_last[act] = self.T_new
        self.T = self.T_new
        self.order = self.order[np.argsort(-self.level[self.order], kind="stable")]
        return w
