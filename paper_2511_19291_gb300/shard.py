"""Partition of independent circuits across ranks.

A batch of circuits (the batched workload: ragged widths and depths, each
with its own parameters and gradient) shards with no data-path collective:
every rank runs its own circuits from start to finish.  The split balances
cost = 2^width x gates (the state bytes one gate-by-gate sweep moves, times
the sweeps), greedily: circuits in decreasing cost order, each to the rank
whose assigned cost is lowest so far (ties to the lower rank).  Every rank
computes the same partition from the same list, so no rank has to send it.

List scheduling of this kind keeps the largest load within the mean load
plus the largest single cost (and within 4/3 of the optimum when sorted,
Graham's bound).
"""
from __future__ import annotations


def circuit_cost(n_qubits: int, n_gates: int) -> int:
    """Cost of one circuit: 2^n_qubits x max(1, n_gates)."""
    if n_qubits < 0 or n_gates < 0:
        raise ValueError("n_qubits and n_gates must be >= 0")
    return (1 << n_qubits) * max(1, n_gates)


def partition(costs, world: int) -> list:
    """Circuit indices per rank (each list ascending): greedy longest-first
    assignment of the costs to `world` ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [int(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be >= 0")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def shard(costs, world: int, rank: int) -> list:
    """The circuit indices rank `rank` of `world` runs."""
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return partition(costs, world)[rank]


def workload_costs(workloads) -> list:
    """circuit_cost of each workload's circuit (objects with .circuit.n_qubits
    and .circuit.gates)."""
    return [circuit_cost(w.circuit.n_qubits, len(w.circuit.gates)) for w in workloads]
