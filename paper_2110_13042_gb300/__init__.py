"""GB300-native (sm_103a) lower-triangle Gram product low(A^T A).

The compute path is the CUDA library ``_build/libata.so`` (C ABI in
``include/ata.h``); :mod:`._binding` is a thin ctypes layer with the same names
that only marshals arguments.  Importing this package does not load the
library; the first call does, and raises if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).  There is no CPU
fallback.
"""
from ._binding import (  # noqa: F401
    ATA_F32, ATA_F32_BF16, ATA_F32_FP8, ATA_F64, ATA_F64_EMU, ATA_PACKED, ATA_TRANS, AtaError, Handle, STATUS, library_path, load,
    plan_blocks, plan_info, status_string, version,
)
