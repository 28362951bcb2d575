"""Seeded synthetic inputs (water boxes and block-sparse matrices) shared by the
oracle and the CUDA path.  Draws inputs only; holds none of the method's arithmetic."""
from .waterbox import BlockMatrix, WaterBox, Hamiltonian, place_waters, decay_matrix, gapped_hamiltonian  # noqa: F401
from .waterbox import overlap_matrix  # noqa: F401
from .configs import Workload, DECAY_32, SIGN_1024, SIGN_4096, SIGN_20736, SUBMATRIX_6192  # noqa: F401
from .configs import batch_seed, batch_systems, small  # noqa: F401
from .configs import build_hamiltonian, build_decay, build_overlap  # noqa: F401
from .random_blocks import random_block_matrix  # noqa: F401
