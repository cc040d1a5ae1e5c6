"""CPU oracle for the open-shell LNO domain (T) energy (arXiv 2311.10048).

TEST INFRASTRUCTURE ONLY.  Plain, slow, float64 PyTorch-on-CPU code that
defines what the GPU library must compute.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library (``paper_2311_10048_gb300``) never does, and this
package imports nothing from the library (inputs arrive as plain arrays).

Modules:
  triples      spin-case per-triplet (T) energy (eq cim_pt_energy), the
               reference for parity; differentiable for the oracle gradient
  spinorbital  the spin-orbital definition by explicit enumeration (tiny)
  closed_shell the textbook closed-shell (T) formula (closed-shell pin)

Pins (tests/test_oracle.py): spin-case == spin-orbital brute force per case;
closed-shell limit == closed-shell formula; W antisymmetry; spin flip;
orbital-energy shift; homogeneity in B and T2; relabelling; gradient against
central finite differences.
"""
from .triples import (CASES, Evaluator, as_tensors, energy, energy_graph,  # noqa: F401
                      n_triplets, triplet_energies, triplets)
