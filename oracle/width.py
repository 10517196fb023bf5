"""Width of the Gaussian energy delta (Eq. (11)) and its adaptive control
(App. C).

Test infrastructure (see ``oracle/__init__``).

Eq. (11) replaces delta(E_in - E_out) by a normalised Gaussian of width
sigma_E (an energy).  App. C uses a fractional width instead,
sigma = w (E_in + E_out) / 2, with E_in and E_out the summed energies of the
initial and final legs of the sample, and adapts w during the run: w is
narrowed when the relative Monte Carlo error is below a lower threshold and
widened when it is above an upper one.

Readings (the paper states neither the error measure nor the step size):
* one w per process, updated after every evaluation of the collision
  integral (one sweep over all tasks) and used from the next evaluation on;
* the relative error of a process is sqrt(sum_t err_t^2) / sum_t |I_t| over
  all its tasks t (grid points, pinned sides, gain and loss), i.e. the
  relative error of its summed rate; no tasks or a zero sum: no update;
* narrowing divides w by a fixed factor, widening multiplies it by that
  factor, and w stays within [width_min, width_max].
"""
import numpy as np

from workloads import WIDTH_ABSOLUTE, WIDTH_ADAPTIVE


def sigma(proc, w, E_sum):
    """Per-sample width: sigma_E, or w (E_in + E_out) / 2 with E_sum the sum
    of all legs' energies (E_in + E_out)."""
    if proc.width_mode == WIDTH_ABSOLUTE:
        return proc.sigma_E
    return 0.5 * w * E_sum


def relative_error(means, errs):
    """sqrt(sum err^2) / sum |mean| of a process's tasks (None: undefined)."""
    means = np.asarray(means, dtype=np.float64)
    errs = np.asarray(errs, dtype=np.float64)
    tot = np.sum(np.abs(means))
    if means.size == 0 or tot == 0.0:
        return None
    return float(np.sqrt(np.sum(errs * errs)) / tot)


def adapt(w, rel, proc):
    """Next w after an evaluation with relative error rel."""
    if proc.width_mode != WIDTH_ADAPTIVE or rel is None:
        return w
    if rel < proc.width_rel_lo:
        w = w / proc.width_factor
    elif rel > proc.width_rel_hi:
        w = w * proc.width_factor
    return min(max(w, proc.width_min), proc.width_max)
