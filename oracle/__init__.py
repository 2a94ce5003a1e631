"""CPU oracle (test infrastructure only; see oracle.py)."""
from .oracle import (adjoint, build, cluster_vectors, eigh_tridiagonal, eigvalsh_tridiagonal,
                     gershgorin_norm, jacobi, kth_eigenvalue, num_threads, split, sturm_count,
                     tridiag_dense)

__all__ = ["adjoint", "build", "cluster_vectors", "eigh_tridiagonal", "eigvalsh_tridiagonal",
           "gershgorin_norm", "jacobi", "kth_eigenvalue", "num_threads", "split", "sturm_count",
           "tridiag_dense"]
