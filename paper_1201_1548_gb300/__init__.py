"""GB300 multi-modular resultant / gcd library: Python binding of the C ABI (include/bsres.h).

The binding only marshals arguments (Python integers <-> two's complement uint32 limbs)
and calls ``libbsres.so``; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the shared library has not been built, or no GPU
is present, the calls raise.

Names follow the C ABI: ``bs_resultant``, ``bs_resultant_batch``, ``bs_resultant_device``,
``bs_uni_resultant_modp``, ``bs_gcd_modp``, ``bs_squarefree_part``, ``bs_prime_table``;
``Context.gcd_z`` / ``Context.modgcd_batch`` wrap ``bs_gcd_z`` / ``bs_modgcd_batch`` and
``Context.serve_start`` / ``submit`` / ``poll`` / ``wait`` / ``serve_stats`` the serving loop.
"""

from ._abi import (  # noqa: F401
    BsError,
    Context,
    bipoly_to_limbs,
    limbs_to_ints,
    ints_to_limbs,
    load_library,
    library_path,
    bs_prime_table,
    bs_plan,
    bs_resultant,
    bs_resultant_batch,
    bs_resultant_bounds,
    bs_resultant_device,
    bs_device_status,
    bs_uni_resultant_modp,
    bs_gcd_modp,
    bs_squarefree_part,
    EXPORTED_SYMBOLS,
    BS_PENDING,
    BS_OK,
    BS_ERR_ARG,
    BS_ERR_NOMEM,
    BS_ERR_UNLUCKY,
    BS_ERR_TIMEOUT,
    BS_ERR_CUDA,
    BS_ERR_ZERO,
    BS_ERR_RANGE,
    BS_ERR_INTERNAL,
    BS_ERR_CAPACITY,
    JOB_RESULTANT,
    JOB_GCD,
    JOB_SQFREE,
)
