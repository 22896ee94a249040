"""GB300-native generalised Brady-Yong fast Hough transform (FHT2DT).

Public API: ``Plan``, ``forward`` and the constants of ``_capi``.  Every step
of the transform runs in ``libfht.so`` (hand-written CUDA for sm_103a); this
package only marshals arguments.
"""
from ._capi import (FHT_CYCLIC, FHT_EXTENDED, FHT_F32_F32, FHT_F64_F64, FHT_I32_I32, FHT_Q0, FHT_Q1,  # noqa: F401
                    FHT_Q2, FHT_Q3, FHT_QALL, FHT_SPLIT_S, FHT_SPLIT_T, FHT_U8_I32, FHTError)
from .fht import HostPipeline, Plan, PlanBuilderPool, PlanCache, forward  # noqa: F401
