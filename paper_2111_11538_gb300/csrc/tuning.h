// Launch shapes per size class, measured on GB300 by
// paper_2111_11538_gb300/autotune.py (which writes this file from the table
// in paper_2111_11538_gb300/data/autotune_gb300.json).
#pragma once
#define FUSED_STARTUP_2D 1
#define FUSED_STARTUP_3D 1
#define PCG_TABLE_2D_F32_LARGE 0
#define PCG_TABLE_2D_F32_SMALL 0
#define PCG_TABLE_2D_F64_LARGE 0
#define PCG_TABLE_2D_F64_SMALL 1
#define PCG_TABLE_3D_F32 0
#define PCG_TABLE_3D_F64 0
#define PCG_TABLE_MG2D_F32_LARGE 1
#define PCG_TABLE_MG2D_F32_SMALL 1
#define PCG_TABLE_MG2D_F64_LARGE 0
#define PCG_TABLE_MG2D_F64_SMALL 1
