//
// Streaming kernels written by hand in PTX: copy a = b, scale a = s*b (mul.rn),
// triad a = b + s*c (fma.rn, one rounding). They are the input of the guard pass, with
// the access order of the hand-fused CUDA kernels: a grid-stride loop over 16-byte units
// (load b, [load c], store a), two units per iteration (i and i + stride, loads first)
// while both exist, then one unit, then the n mod 4 tail elements with 4-byte accesses by
// the first threads of the grid. Parameters: a, b, c (u64 device addresses), n (u64
// element count), s (f32).
//
.version 9.0
.target sm_103a
.address_size 64

.visible .entry agile_ptx_copy(
	.param .u64 p_a,
	.param .u64 p_b,
	.param .u64 p_c,
	.param .u64 p_n,
	.param .f32 p_s
)
{
	.reg .pred %p<4>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<24>;
	.reg .f32 %f<32>;

	ld.param.u64 %rd1, [p_a];
	ld.param.u64 %rd2, [p_b];
	ld.param.u64 %rd3, [p_c];
	ld.param.u64 %rd4, [p_n];
	ld.param.f32 %f15, [p_s];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shl.b64 %rd16, %rd7, 4;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
$PAIR:
	add.s64 %rd17, %rd9, %rd7;
	setp.ge.u64 %p1, %rd17, %rd8;
	@%p1 bra $ONE;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	add.s64 %rd18, %rd11, %rd16;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	ld.global.v4.f32 {%f16, %f17, %f18, %f19}, [%rd18];
	mov.f32 %f24, %f1;
	mov.f32 %f25, %f2;
	mov.f32 %f26, %f3;
	mov.f32 %f27, %f4;
	mov.f32 %f28, %f16;
	mov.f32 %f29, %f17;
	mov.f32 %f30, %f18;
	mov.f32 %f31, %f19;
	add.s64 %rd12, %rd1, %rd10;
	add.s64 %rd20, %rd12, %rd16;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
	st.global.v4.f32 [%rd20], {%f28, %f29, %f30, %f31};
	add.s64 %rd9, %rd17, %rd7;
	bra.uni $PAIR;
$ONE:
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	mov.f32 %f24, %f1;
	mov.f32 %f25, %f2;
	mov.f32 %f26, %f3;
	mov.f32 %f27, %f4;
	add.s64 %rd12, %rd1, %rd10;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
$TAIL:
	and.b64 %rd14, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd14;
	@%p2 bra $DONE;
	shl.b64 %rd15, %rd8, 2;
	add.s64 %rd15, %rd15, %rd5;
	shl.b64 %rd15, %rd15, 2;
	add.s64 %rd11, %rd2, %rd15;
	ld.global.f32 %f9, [%rd11];
	add.s64 %rd12, %rd1, %rd15;
	st.global.f32 [%rd12], %f9;
$DONE:
	ret;
}

.visible .entry agile_ptx_scale(
	.param .u64 p_a,
	.param .u64 p_b,
	.param .u64 p_c,
	.param .u64 p_n,
	.param .f32 p_s
)
{
	.reg .pred %p<4>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<24>;
	.reg .f32 %f<32>;

	ld.param.u64 %rd1, [p_a];
	ld.param.u64 %rd2, [p_b];
	ld.param.u64 %rd3, [p_c];
	ld.param.u64 %rd4, [p_n];
	ld.param.f32 %f15, [p_s];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shl.b64 %rd16, %rd7, 4;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
$PAIR:
	add.s64 %rd17, %rd9, %rd7;
	setp.ge.u64 %p1, %rd17, %rd8;
	@%p1 bra $ONE;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	add.s64 %rd18, %rd11, %rd16;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	ld.global.v4.f32 {%f16, %f17, %f18, %f19}, [%rd18];
	mul.rn.f32 %f24, %f15, %f1;
	mul.rn.f32 %f25, %f15, %f2;
	mul.rn.f32 %f26, %f15, %f3;
	mul.rn.f32 %f27, %f15, %f4;
	mul.rn.f32 %f28, %f15, %f16;
	mul.rn.f32 %f29, %f15, %f17;
	mul.rn.f32 %f30, %f15, %f18;
	mul.rn.f32 %f31, %f15, %f19;
	add.s64 %rd12, %rd1, %rd10;
	add.s64 %rd20, %rd12, %rd16;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
	st.global.v4.f32 [%rd20], {%f28, %f29, %f30, %f31};
	add.s64 %rd9, %rd17, %rd7;
	bra.uni $PAIR;
$ONE:
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	mul.rn.f32 %f24, %f15, %f1;
	mul.rn.f32 %f25, %f15, %f2;
	mul.rn.f32 %f26, %f15, %f3;
	mul.rn.f32 %f27, %f15, %f4;
	add.s64 %rd12, %rd1, %rd10;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
$TAIL:
	and.b64 %rd14, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd14;
	@%p2 bra $DONE;
	shl.b64 %rd15, %rd8, 2;
	add.s64 %rd15, %rd15, %rd5;
	shl.b64 %rd15, %rd15, 2;
	add.s64 %rd11, %rd2, %rd15;
	ld.global.f32 %f9, [%rd11];
	mul.rn.f32 %f9, %f15, %f9;
	add.s64 %rd12, %rd1, %rd15;
	st.global.f32 [%rd12], %f9;
$DONE:
	ret;
}

.visible .entry agile_ptx_triad(
	.param .u64 p_a,
	.param .u64 p_b,
	.param .u64 p_c,
	.param .u64 p_n,
	.param .f32 p_s
)
{
	.reg .pred %p<4>;
	.reg .b32 %r<6>;
	.reg .b64 %rd<24>;
	.reg .f32 %f<32>;

	ld.param.u64 %rd1, [p_a];
	ld.param.u64 %rd2, [p_b];
	ld.param.u64 %rd3, [p_c];
	ld.param.u64 %rd4, [p_n];
	ld.param.f32 %f15, [p_s];
	mov.u32 %r1, %ctaid.x;
	mov.u32 %r2, %ntid.x;
	mov.u32 %r3, %tid.x;
	mov.u32 %r4, %nctaid.x;
	mul.wide.u32 %rd5, %r1, %r2;
	cvt.u64.u32 %rd6, %r3;
	add.s64 %rd5, %rd5, %rd6;
	mul.wide.u32 %rd7, %r4, %r2;
	shl.b64 %rd16, %rd7, 4;
	shr.u64 %rd8, %rd4, 2;
	mov.b64 %rd9, %rd5;
$PAIR:
	add.s64 %rd17, %rd9, %rd7;
	setp.ge.u64 %p1, %rd17, %rd8;
	@%p1 bra $ONE;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	add.s64 %rd18, %rd11, %rd16;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	ld.global.v4.f32 {%f16, %f17, %f18, %f19}, [%rd18];
	add.s64 %rd13, %rd3, %rd10;
	add.s64 %rd19, %rd13, %rd16;
	ld.global.v4.f32 {%f5, %f6, %f7, %f8}, [%rd13];
	ld.global.v4.f32 {%f20, %f21, %f22, %f23}, [%rd19];
	fma.rn.f32 %f24, %f15, %f5, %f1;
	fma.rn.f32 %f25, %f15, %f6, %f2;
	fma.rn.f32 %f26, %f15, %f7, %f3;
	fma.rn.f32 %f27, %f15, %f8, %f4;
	fma.rn.f32 %f28, %f15, %f20, %f16;
	fma.rn.f32 %f29, %f15, %f21, %f17;
	fma.rn.f32 %f30, %f15, %f22, %f18;
	fma.rn.f32 %f31, %f15, %f23, %f19;
	add.s64 %rd12, %rd1, %rd10;
	add.s64 %rd20, %rd12, %rd16;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
	st.global.v4.f32 [%rd20], {%f28, %f29, %f30, %f31};
	add.s64 %rd9, %rd17, %rd7;
	bra.uni $PAIR;
$ONE:
	setp.ge.u64 %p1, %rd9, %rd8;
	@%p1 bra $TAIL;
	shl.b64 %rd10, %rd9, 4;
	add.s64 %rd11, %rd2, %rd10;
	ld.global.v4.f32 {%f1, %f2, %f3, %f4}, [%rd11];
	add.s64 %rd13, %rd3, %rd10;
	ld.global.v4.f32 {%f5, %f6, %f7, %f8}, [%rd13];
	fma.rn.f32 %f24, %f15, %f5, %f1;
	fma.rn.f32 %f25, %f15, %f6, %f2;
	fma.rn.f32 %f26, %f15, %f7, %f3;
	fma.rn.f32 %f27, %f15, %f8, %f4;
	add.s64 %rd12, %rd1, %rd10;
	st.global.v4.f32 [%rd12], {%f24, %f25, %f26, %f27};
$TAIL:
	and.b64 %rd14, %rd4, 3;
	setp.ge.u64 %p2, %rd5, %rd14;
	@%p2 bra $DONE;
	shl.b64 %rd15, %rd8, 2;
	add.s64 %rd15, %rd15, %rd5;
	shl.b64 %rd15, %rd15, 2;
	add.s64 %rd11, %rd2, %rd15;
	ld.global.f32 %f9, [%rd11];
	add.s64 %rd13, %rd3, %rd15;
	ld.global.f32 %f10, [%rd13];
	fma.rn.f32 %f9, %f15, %f10, %f9;
	add.s64 %rd12, %rd1, %rd15;
	st.global.f32 [%rd12], %f9;
$DONE:
	ret;
}
