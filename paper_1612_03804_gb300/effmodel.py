"""Interaction classes of the effective Ising model (Eq. 2).

H_eff = E0 + sum_c J_c f_c(C), f_c(C) = sum_x sum_{o in c} s_x s_{x+o}, with
x = (site, slice) on the periodic Lx x Ly x M space-time lattice and each
class c a set of offsets o = (dx, dy, dtau) related by the lattice
symmetries ("Formalism of SLDQMC": symmetries reduce the couplings to a few
independent ones; gamma is their range).  Every unordered pair {x, x+o}
appears once: a class lists one of o and -o.

Two families:
  CLASSES_4  -- J1 (nearest neighbours), J2 (diagonal), J3 (distance 2 on
                an axis) at equal slice, and J_tau (same site, adjacent
                slices): the model of the 16x16 workload.
  paper_classes() -- the model of "Results": spatial shells up to the 2nd
                neighbour, temporal couplings up to |dtau| = 10 (= M/2 at
                M = 20), and spatio-temporal couplings, 16 in all.  The
                paper names the counts (2 spatial, 10 temporal, 4
                spatio-temporal) but not the shapes of the last four; they
                are read here as the two spatial shells at |dtau| = 1 and 2.
range scans -- the two 1 - R^2 curves of "Results": the temporal range
                with the spatial range fixed at nearest neighbours, and the
                spatial range with the temporal range fixed at 10.
"""

# spatial shells of the square lattice by distance: 1, sqrt 2, 2, sqrt 5, sqrt 8, 3
SHELLS = [
    [(1, 0), (0, 1)],
    [(1, 1), (1, -1)],
    [(2, 0), (0, 2)],
    [(2, 1), (1, 2), (2, -1), (1, -2)],
    [(2, 2), (2, -2)],
    [(3, 0), (0, 3)],
]

CLASSES_4 = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]


def spatial_class(shell):
    """Equal-slice pairs at the shell's distance."""
    return [(dx, dy, 0) for dx, dy in SHELLS[shell - 1]]


def temporal_class(k):
    """Same-site pairs k slices apart."""
    return [(0, 0, k)]


def spatio_temporal_class(shell, k):
    """Pairs at the shell's spatial distance and k > 0 slices apart: (o, k)
    and (-o, k) are different unordered pairs, so both signs appear."""
    out = []
    for dx, dy in SHELLS[shell - 1]:
        out.append((dx, dy, k))
        out.append((-dx, -dy, k))
    return out


def paper_classes(n_shell=2, n_time=10, st_shells=2, st_times=2):
    """The effective model of "Results": n_shell spatial + n_time temporal +
    st_shells * st_times spatio-temporal classes (16 with the defaults)."""
    cls = [spatial_class(s) for s in range(1, n_shell + 1)]
    cls += [temporal_class(k) for k in range(1, n_time + 1)]
    cls += [spatio_temporal_class(s, k) for s in range(1, st_shells + 1) for k in range(1, st_times + 1)]
    return cls


def class_names(n_shell=2, n_time=10, st_shells=2, st_times=2):
    names = [f"space{s}" for s in range(1, n_shell + 1)]
    names += [f"time{k}" for k in range(1, n_time + 1)]
    names += [f"space{s}_time{k}" for s in range(1, st_shells + 1) for k in range(1, st_times + 1)]
    return names


def temporal_range_scan(max_k=10):
    """Class sets for the temporal-range curve: nearest-neighbour space plus
    temporal couplings up to k, for k = 1..max_k."""
    return [(k, [spatial_class(1)] + [temporal_class(j) for j in range(1, k + 1)]) for k in range(1, max_k + 1)]


def spatial_range_scan(max_shell=5, n_time=10):
    """Class sets for the spatial-range curve: temporal couplings up to
    n_time plus spatial shells up to s, for s = 1..max_shell."""
    return [(s, [spatial_class(j) for j in range(1, s + 1)] + [temporal_class(k) for k in range(1, n_time + 1)])
            for s in range(1, max_shell + 1)]


def n_offsets(classes):
    return sum(len(c) for c in classes)
