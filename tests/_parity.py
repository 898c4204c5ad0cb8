"""Helpers shared by the GPU parity tests (no method arithmetic)."""
import numpy as np

# A bond decision of a free FP32 run may differ from the oracle's only where
# the oracle's uniform or gap lay this close to its threshold (the FP32
# trajectory tolerance, lattice units / probability).
NEAR_TIE = 1e-4


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def bonds_every_step(pairs, advance, steps, label, pid=0):
    """Advances every (oracle, gpu sim) pair one step at a time (advance()
    steps the GPU side of all of them) and compares the bond flags at every
    step.  A difference is accepted only at a step where the oracle logged a
    near tie; afterwards that pair's flags are no longer compared.  Returns
    per pair (first divergence step or None, final Hamming distance)."""
    first = [None] * len(pairs)
    for t in range(steps):
        for o, _ in pairs:
            o.step(1)
        advance()
        for j, (o, g) in enumerate(pairs):
            if first[j] is not None:
                continue
            bo, _ = o.bonds(pid)
            bg, _ = g.bonds(pid)
            if not np.array_equal(bo, bg):
                first[j] = t + 1
                st = o.particle(pid)
                assert min(st["margin_p"], st["margin_gap"]) < NEAR_TIE, (
                    f"{label}[{j}]: bond flags differ at step {t + 1} without a near tie "
                    f"(|U-P| {st['margin_p']:.3g}, |gap-y_cr| {st['margin_gap']:.3g})")
    out = []
    for j, (o, g) in enumerate(pairs):
        ham = int((o.bonds(pid)[0] != g.bonds(pid)[0]).sum())
        print(f"{label}[{j}]: first bond divergence {first[j]}, Hamming distance {ham} "
              f"after {steps} steps")
        out.append((first[j], ham))
    return out
