"""Identical-particle decomposition (Sec. 2C) and particle roles (App. A).

Test infrastructure (see ``oracle/__init__``).

A *side integral* is C_{n_alpha} of Eq. (7) for one process, one observed
species a and one side S (the side holding the observed leg).  Its result
enters C_a with the multiplicity n_S^a, the number of times a appears on S
(Eq. (7)).  For a process whose initial and final species multisets are equal
(the symmetric case of Eq. (8)) only the initial side is evaluated, with
multiplicity n_in^a.  Readings for cases the paper does not spell out:
  * AB -> AB style processes (equal multisets, several species) follow the
    same rule: one side per observed species, multiplicity n_in^a;
  * AA -> BB style processes (n_in = n_out, different multisets) take both
    sides, like asymmetric processes.

Roles inside a side integral (App. A):
  * observed: the lowest index of species a on side S;
  * conserved: if n_in != n_out, the lowest index other than the observed one
    on the side with fewer legs; if that side holds only the observed leg,
    the lowest index on the opposite side; if n_in == n_out, the lowest
    index other than the observed one on the observed side (with the same
    fallback);
  * integrated: the remaining n - 2 legs in index order, each with three
    VEGAS dimensions (r, theta, phi) in that order.

A process may restrict the side integrals evaluated (``sides`` = 1: those
with the observed leg initial, 2: final), as in the paper's comparison of
C = 2 C_2 + 3 C_3 with C_3 alone (Sec. 5D).

Task enumeration (shared convention with the CUDA library): side integrals
are ordered by process, then side (initial before final), then species index;
task id = (side_integral * n_grid + grid_point) * 2 + term, term 0 = gain and
1 = loss (Sec. 2D: separate integrators for gain and loss).
"""
from dataclasses import dataclass
from typing import List, Tuple

SIDE_IN = 0
SIDE_OUT = 1


@dataclass(frozen=True)
class SideIntegral:
    process: int
    side: int                 # side of the observed leg
    species: int              # observed species a
    mult: int                 # n_S^a of Eq. (7)
    legs: Tuple[int, ...]     # species of legs 0..n-1 (initial legs first)
    n_in: int
    obs: int
    cons: int
    integrated: Tuple[int, ...]

    @property
    def n(self):
        return len(self.legs)

    @property
    def dim(self):
        return 3 * (self.n - 2)

    def is_in(self, k):
        return k < self.n_in


def roles(n_in, n_out, obs):
    """(conserved index, integrated indices) for an observed leg (App. A)."""
    n = n_in + n_out
    in_side = list(range(n_in))
    out_side = list(range(n_in, n))
    obs_in = obs < n_in
    if n_in != n_out:
        first = in_side if n_in < n_out else out_side
    else:
        first = in_side if obs_in else out_side
    other = out_side if first is in_side else in_side
    cand = [k for k in first if k != obs]
    if not cand:
        cand = [k for k in other if k != obs]
    cons = cand[0]
    integrated = tuple(k for k in range(n) if k not in (obs, cons))
    return cons, integrated


def side_integrals(problem) -> List[SideIntegral]:
    """All side integrals of a problem in task-enumeration order."""
    out = []
    for ip, proc in enumerate(problem.processes):
        sp_in, sp_out = tuple(proc.species_in), tuple(proc.species_out)
        n_in, n_out = len(sp_in), len(sp_out)
        if n_in + n_out < 3:
            raise ValueError("a process needs at least three legs")
        legs = sp_in + sp_out
        symmetric = sorted(sp_in) == sorted(sp_out)
        sides = [SIDE_IN] if symmetric else [SIDE_IN, SIDE_OUT]
        keep = getattr(proc, "sides", 0)           # 1: initial side only, 2: final side only
        if keep:
            sides = [s for s in sides if s == keep - 1]
        for side in sides:
            side_species = sp_in if side == SIDE_IN else sp_out
            offset = 0 if side == SIDE_IN else n_in
            for a in sorted(set(side_species)):
                obs = offset + side_species.index(a)
                cons, integ = roles(n_in, n_out, obs)
                out.append(SideIntegral(ip, side, a, side_species.count(a), legs,
                                        n_in, obs, cons, integ))
    return out


def task_id(side_integral_index, grid_point, term, n_grid):
    return (side_integral_index * n_grid + grid_point) * 2 + term
