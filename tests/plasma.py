"""Test inputs: the seeded drifting pair plasmas of `workloads`, with the particle arrays drawn
by the FP64 oracle's App. D loader (oracle.load_drifting) on the host.  The GPU and the oracle
are then handed the very same arrays; the library's own device loader is tested against the
oracle's in test_gpu_loader.py."""
import dataclasses

import oracle
import workloads


def fill(wl, first=0, count=None):
    """The workload with every species' x (dim, n) and u (3, n) as numpy FP64 arrays (particles
    first .. first + count - 1 of each species when given)."""
    species = []
    for i, s in enumerate(wl.species):
        x, u, failed = oracle.load_drifting(wl.grid, wl.dx, s.per_cell, wl.gamma, wl.u_th,
                                            wl.theta, wl.seed, wl.run, i, s.pos_species,
                                            first=first, count=count)
        assert failed == 0
        species.append(dataclasses.replace(s, x=x, u=u))
    return dataclasses.replace(wl, species=species)


def pair_plasma(*args, **kw):
    return fill(workloads.pair_plasma(*args, **kw))


def config_small(**kw):
    return fill(workloads.config_small(**kw))


def config_large(**kw):
    return fill(workloads.config_large(**kw))
