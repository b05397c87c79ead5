//
// Irregular kernels written by hand in PTX, the input of the guard pass: gather
// out[i] = T[idx[i]], scatter T[idx[i]] = (float)(idx[i] & 0xFFFFFF), histogram
// bins[idx[i]] += 1 (red.global.add). Same access order as the hand-fused CUDA kernels:
// per group of four elements two 16-byte index loads, four element accesses and (gather)
// a 16-byte output store; then the n mod 4 tail elements one by one. Parameters: idx
// (u64 address of int64 offsets), base (u64 address of T or the bins), out (u64),
// n (u64 elements).
//
.version 9.0
.target sm_103a
.address_size 64

.visible .entry agile_ptx_gather(
	.param .u64 p_idx,
	.param .u64 p_base,
	.param .u64 p_out,
	.param .u64 p_n
)
{
	.reg .pred %p<3>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<32>;
	.reg .f32 %f<8>;

	ld.param.u64 %rd1, [p_idx];
	ld.param.u64 %rd2, [p_base];
	ld.param.u64 %rd3, [p_out];
	ld.param.u64 %rd4, [p_n];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
$LOOP:
	shl.b64 %rd10, %rd9, 5;
	add.s64 %rd11, %rd1, %rd10;
	ld.global.v2.u64 {%rd12, %rd13}, [%rd11];
	ld.global.v2.u64 {%rd14, %rd15}, [%rd11+16];
	shl.b64 %rd16, %rd12, 2;
	add.s64 %rd16, %rd2, %rd16;
	ld.global.f32 %f1, [%rd16];
	shl.b64 %rd17, %rd13, 2;
	add.s64 %rd17, %rd2, %rd17;
	ld.global.f32 %f2, [%rd17];
	shl.b64 %rd18, %rd14, 2;
	add.s64 %rd18, %rd2, %rd18;
	ld.global.f32 %f3, [%rd18];
	shl.b64 %rd19, %rd15, 2;
	add.s64 %rd19, %rd2, %rd19;
	ld.global.f32 %f4, [%rd19];
	shl.b64 %rd20, %rd9, 4;
	add.s64 %rd20, %rd3, %rd20;
	st.global.v4.f32 [%rd20], {%f1, %f2, %f3, %f4};
	add.s64 %rd9, %rd9, %rd7;
	setp.lt.u64 %p1, %rd9, %rd8;
	@%p1 bra $LOOP;
$TAIL:
	and.b64 %rd21, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd21;
	@%p2 bra $DONE;
	shl.b64 %rd22, %rd8, 2;
	add.s64 %rd22, %rd22, %rd5;
	shl.b64 %rd23, %rd22, 3;
	add.s64 %rd23, %rd1, %rd23;
	ld.global.u64 %rd24, [%rd23];
	shl.b64 %rd16, %rd24, 2;
	add.s64 %rd16, %rd2, %rd16;
	ld.global.f32 %f1, [%rd16];
	shl.b64 %rd25, %rd22, 2;
	add.s64 %rd25, %rd3, %rd25;
	st.global.f32 [%rd25], %f1;
$DONE:
	ret;
}

.visible .entry agile_ptx_scatter(
	.param .u64 p_idx,
	.param .u64 p_base,
	.param .u64 p_out,
	.param .u64 p_n
)
{
	.reg .pred %p<3>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<32>;
	.reg .f32 %f<8>;

	ld.param.u64 %rd1, [p_idx];
	ld.param.u64 %rd2, [p_base];
	ld.param.u64 %rd3, [p_out];
	ld.param.u64 %rd4, [p_n];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
$LOOP:
	shl.b64 %rd10, %rd9, 5;
	add.s64 %rd11, %rd1, %rd10;
	ld.global.v2.u64 {%rd12, %rd13}, [%rd11];
	ld.global.v2.u64 {%rd14, %rd15}, [%rd11+16];
	shl.b64 %rd16, %rd12, 2;
	add.s64 %rd16, %rd2, %rd16;
	and.b64 %rd30, %rd12, 16777215;
	cvt.rn.f32.u64 %f1, %rd30;
	st.global.f32 [%rd16], %f1;
	shl.b64 %rd17, %rd13, 2;
	add.s64 %rd17, %rd2, %rd17;
	and.b64 %rd30, %rd13, 16777215;
	cvt.rn.f32.u64 %f2, %rd30;
	st.global.f32 [%rd17], %f2;
	shl.b64 %rd18, %rd14, 2;
	add.s64 %rd18, %rd2, %rd18;
	and.b64 %rd30, %rd14, 16777215;
	cvt.rn.f32.u64 %f3, %rd30;
	st.global.f32 [%rd18], %f3;
	shl.b64 %rd19, %rd15, 2;
	add.s64 %rd19, %rd2, %rd19;
	and.b64 %rd30, %rd15, 16777215;
	cvt.rn.f32.u64 %f4, %rd30;
	st.global.f32 [%rd19], %f4;
	add.s64 %rd9, %rd9, %rd7;
	setp.lt.u64 %p1, %rd9, %rd8;
	@%p1 bra $LOOP;
$TAIL:
	and.b64 %rd21, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd21;
	@%p2 bra $DONE;
	shl.b64 %rd22, %rd8, 2;
	add.s64 %rd22, %rd22, %rd5;
	shl.b64 %rd23, %rd22, 3;
	add.s64 %rd23, %rd1, %rd23;
	ld.global.u64 %rd24, [%rd23];
	shl.b64 %rd16, %rd24, 2;
	add.s64 %rd16, %rd2, %rd16;
	and.b64 %rd30, %rd24, 16777215;
	cvt.rn.f32.u64 %f1, %rd30;
	st.global.f32 [%rd16], %f1;
$DONE:
	ret;
}

.visible .entry agile_ptx_hist(
	.param .u64 p_idx,
	.param .u64 p_base,
	.param .u64 p_out,
	.param .u64 p_n
)
{
	.reg .pred %p<3>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<32>;
	.reg .f32 %f<8>;

	ld.param.u64 %rd1, [p_idx];
	ld.param.u64 %rd2, [p_base];
	ld.param.u64 %rd3, [p_out];
	ld.param.u64 %rd4, [p_n];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
$LOOP:
	shl.b64 %rd10, %rd9, 5;
	add.s64 %rd11, %rd1, %rd10;
	ld.global.v2.u64 {%rd12, %rd13}, [%rd11];
	ld.global.v2.u64 {%rd14, %rd15}, [%rd11+16];
	shl.b64 %rd16, %rd12, 2;
	add.s64 %rd16, %rd2, %rd16;
	red.global.add.u32 [%rd16], 1;
	shl.b64 %rd17, %rd13, 2;
	add.s64 %rd17, %rd2, %rd17;
	red.global.add.u32 [%rd17], 1;
	shl.b64 %rd18, %rd14, 2;
	add.s64 %rd18, %rd2, %rd18;
	red.global.add.u32 [%rd18], 1;
	shl.b64 %rd19, %rd15, 2;
	add.s64 %rd19, %rd2, %rd19;
	red.global.add.u32 [%rd19], 1;
	add.s64 %rd9, %rd9, %rd7;
	setp.lt.u64 %p1, %rd9, %rd8;
	@%p1 bra $LOOP;
$TAIL:
	and.b64 %rd21, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd21;
	@%p2 bra $DONE;
	shl.b64 %rd22, %rd8, 2;
	add.s64 %rd22, %rd22, %rd5;
	shl.b64 %rd23, %rd22, 3;
	add.s64 %rd23, %rd1, %rd23;
	ld.global.u64 %rd24, [%rd23];
	shl.b64 %rd16, %rd24, 2;
	add.s64 %rd16, %rd2, %rd16;
	red.global.add.u32 [%rd16], 1;
$DONE:
	ret;
}
